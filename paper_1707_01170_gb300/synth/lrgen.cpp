// Seeded synthetic LR-spline volumes: structured-mesh local refinement.
//
// This is INPUT construction, shared by the CPU oracle tests and the CUDA
// path; it evaluates nothing of the rendering method (no element look-up,
// no Bezier conversion, no ray marching).  It produces the data the paper's
// method consumes: a box partition of [0,1]^3 into elements and a set of LR
// B-splines, each a product of three univariate B-splines on local knot
// vectors, with scale factors gamma that keep a partition of unity (Eq. 2).
//
// LR B-splines come from local refinements of a tensor-product mesh: each
// B-spline that a new mesh plane cuts clean through is split, and this is
// repeated until no mesh plane cuts through any support (Sec. 3.1).  The
// refinement strategy used here is the structured
// mesh one: every B-spline whose support meets a marked element gets its
// support halved in every knot interval, in all three directions, by mesh
// rectangles spanning the support; then every B-spline whose support is
// traversed by a mesh plane is split by single-knot insertion,
//   B[xi] = a1 * B[xi'_0..p+1] + a2 * B[xi'_1..p+2],
// with a1 = min(1, (t - xi_0)/(xi_p - xi_0)), a2 = min(1, (xi_{p+1} - t)/(xi_{p+1} - xi_1)),
// until no split is possible.  Duplicate B-splines merge by summing the
// gamma-weighted terms, so sum_i gamma_i N_i stays 1.
//
// All coordinates are integers on a grid of resolution G_a = n_a * 2^levels
// per axis, so every knot and every element face is exact.
//
// The random source is std::mt19937_64 (its output sequence is fixed by the
// C++ standard); uniforms are (x >> 11) * 2^-53.

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <random>
#include <unordered_map>
#include <vector>

namespace {

constexpr int kMaxP = 4;
constexpr int kKey = 3 * (kMaxP + 2);

struct Box {
  int32_t lo[3], hi[3];
};

using Key = std::array<int32_t, kKey>;

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int32_t v : k) {
      h ^= (uint64_t)(uint32_t)v;
      h *= 1099511628211ull;
    }
    return (size_t)(h ^ (h >> 29));
  }
};

struct BSpl {
  Key k;            // knots of axis a at k[a*(kMaxP+2) + j], j = 0..p_a+1; unused = -1
  double gamma;
  double gc[3];     // gamma * coefficient (carried through splits)
  bool alive;
};

struct Gen {
  int p[3];
  int n[3];
  int levels;
  int G[3];
  int nc;
  std::vector<Box> el;
  std::vector<BSpl> bs;
  std::unordered_map<Key, int64_t, KeyHash> index;
  // element bucket grid (stale entries allowed; filtered at query)
  int nb[3];
  int bw[3];  // bucket width in grid units
  std::vector<std::vector<int32_t>> buckets;
  std::vector<uint32_t> stamp;
  uint32_t cur_stamp = 0;
  int last_error = 0;

  int32_t kn(const BSpl& b, int a, int j) const { return b.k[a * (kMaxP + 2) + j]; }

  void bucket_range(const Box& q, int lo[3], int hi[3]) const {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::max(0, q.lo[a] / bw[a]);
      hi[a] = std::min(nb[a] - 1, (q.hi[a] - 1) / bw[a]);
    }
  }

  void add_to_buckets(int32_t e) {
    int lo[3], hi[3];
    bucket_range(el[e], lo, hi);
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x)
          buckets[((size_t)z * nb[1] + y) * nb[0] + x].push_back(e);
  }

  void rebuild_buckets() {
    for (auto& b : buckets) b.clear();
    for (int32_t e = 0; e < (int32_t)el.size(); ++e) add_to_buckets(e);
  }

  static bool overlaps(const Box& a, const Box& b) {
    for (int d = 0; d < 3; ++d)
      if (!(a.lo[d] < b.hi[d] && b.lo[d] < a.hi[d])) return false;
    return true;
  }

  // Elements overlapping q with positive volume.
  void query(const Box& q, std::vector<int32_t>& out) {
    out.clear();
    if (stamp.size() < el.size()) stamp.resize(el.size() * 2 + 16, 0);
    ++cur_stamp;
    if (cur_stamp == 0) {
      std::fill(stamp.begin(), stamp.end(), 0);
      cur_stamp = 1;
    }
    int lo[3], hi[3];
    bucket_range(q, lo, hi);
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x)
          for (int32_t e : buckets[((size_t)z * nb[1] + y) * nb[0] + x]) {
            if (stamp[e] == cur_stamp) continue;
            stamp[e] = cur_stamp;
            if (overlaps(el[e], q)) out.push_back(e);
          }
  }

  Box support(const BSpl& b) const {
    Box s;
    for (int a = 0; a < 3; ++a) {
      s.lo[a] = kn(b, a, 0);
      s.hi[a] = kn(b, a, p[a] + 1);
    }
    return s;
  }

  int64_t add_bspline(const Key& k, double gamma, const double* gc) {
    auto it = index.find(k);
    if (it != index.end() && bs[it->second].alive) {
      BSpl& b = bs[it->second];
      b.gamma += gamma;
      for (int c = 0; c < 3; ++c) b.gc[c] += gc[c];
      return it->second;
    }
    BSpl b;
    b.k = k;
    b.gamma = gamma;
    for (int c = 0; c < 3; ++c) b.gc[c] = gc[c];
    b.alive = true;
    bs.push_back(b);
    int64_t id = (int64_t)bs.size() - 1;
    index[k] = id;
    return id;
  }

  void init(const int* deg, const int* nbase, int lev, int ncomp) {
    for (int a = 0; a < 3; ++a) {
      p[a] = deg[a];
      n[a] = nbase[a];
      G[a] = n[a] << lev;
    }
    levels = lev;
    nc = ncomp;
    // uniform tensor-product elements
    el.clear();
    int h[3] = {G[0] / n[0], G[1] / n[1], G[2] / n[2]};
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          Box b;
          b.lo[0] = i * h[0]; b.hi[0] = (i + 1) * h[0];
          b.lo[1] = j * h[1]; b.hi[1] = (j + 1) * h[1];
          b.lo[2] = k * h[2]; b.hi[2] = (k + 1) * h[2];
          el.push_back(b);
        }
    // bucket grid: about 64 buckets per axis at most, at least 1 grid unit wide
    for (int a = 0; a < 3; ++a) {
      nb[a] = std::min(G[a], 32);
      bw[a] = (G[a] + nb[a] - 1) / nb[a];
      nb[a] = (G[a] + bw[a] - 1) / bw[a];
    }
    buckets.assign((size_t)nb[0] * nb[1] * nb[2], {});
    rebuild_buckets();
    // open (clamped) global knot vectors; local vectors are windows of p+2 knots
    std::vector<int32_t> U[3];
    for (int a = 0; a < 3; ++a) {
      for (int r = 0; r < p[a]; ++r) U[a].push_back(0);
      for (int i = 0; i <= n[a]; ++i) U[a].push_back(i * h[a]);
      for (int r = 0; r < p[a]; ++r) U[a].push_back(G[a]);
    }
    bs.clear();
    index.clear();
    int l[3] = {n[0] + p[0], n[1] + p[1], n[2] + p[2]};
    double zero[3] = {0, 0, 0};
    for (int k = 0; k < l[2]; ++k)
      for (int j = 0; j < l[1]; ++j)
        for (int i = 0; i < l[0]; ++i) {
          Key key;
          key.fill(-1);
          int idx[3] = {i, j, k};
          for (int a = 0; a < 3; ++a)
            for (int r = 0; r <= p[a] + 1; ++r) key[a * (kMaxP + 2) + r] = U[a][idx[a] + r];
          add_bspline(key, 1.0, zero);
        }
  }

  // Split element boxes straddling the plane x_a = t inside the rectangle
  // spanned (in the other two axes) by box r.
  void insert_rectangle(int a, int32_t t, const Box& r) {
    Box q = r;
    q.lo[a] = t - 1;
    q.hi[a] = t + 1;
    std::vector<int32_t> hit;
    query(q, hit);
    for (int32_t e : hit) {
      Box b = el[e];
      if (!(b.lo[a] < t && t < b.hi[a])) continue;
      Box b1 = b, b2 = b;
      b1.hi[a] = t;
      b2.lo[a] = t;
      el[e] = b1;
      el.push_back(b2);
      add_to_buckets((int32_t)el.size() - 1);
    }
  }

  // Knots t of axis a whose mesh plane traverses the support of b (no element
  // inside the support straddles x_a = t) and that are not knots of b yet.
  void traversing_knots(const BSpl& b, const std::vector<int32_t>& inside, int a,
                        std::vector<int32_t>& out) {
    out.clear();
    Box s = support(b);
    const int pa = p[a];
    std::vector<int32_t> cand;
    for (int32_t e : inside) {
      int32_t t = el[e].lo[a];
      if (t <= s.lo[a] || t >= s.hi[a]) continue;
      bool isknot = false;
      for (int j = 0; j <= pa + 1; ++j) isknot |= (kn(b, a, j) == t);
      if (!isknot) cand.push_back(t);
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int32_t t : cand) {
      bool straddled = false;
      for (int32_t e : inside)
        if (el[e].lo[a] < t && t < el[e].hi[a]) {
          straddled = true;
          break;
        }
      if (!straddled) out.push_back(t);
    }
  }

  static int64_t volume(const Box& s) {
    return (int64_t)(s.hi[0] - s.lo[0]) * (s.hi[1] - s.lo[1]) * (s.hi[2] - s.lo[2]);
  }

  // Split B-splines until all have minimal support.  Every split sends weight
  // only to B-splines of strictly smaller support, so taking B-splines in
  // decreasing support volume handles each one once, after all its incoming
  // weight has arrived.  All traversing knots of one axis are inserted
  // together by repeated single-knot insertion of the univariate factor.
  int closure() {
    std::vector<std::pair<int64_t, int64_t>> heap;  // (volume, id)
    for (size_t id = 0; id < bs.size(); ++id)
      if (bs[id].alive) heap.push_back({volume(support(bs[id])), (int64_t)id});
    std::make_heap(heap.begin(), heap.end());
    std::vector<int32_t> inside, knots;
    struct Win {
      int32_t k[kMaxP + 2];
      double w;
    };
    std::vector<Win> cur, nxt;
    while (!heap.empty()) {
      std::pop_heap(heap.begin(), heap.end());
      int64_t id = heap.back().second;
      heap.pop_back();
      if (!bs[id].alive) continue;
      Box s = support(bs[id]);
      query(s, inside);
      for (int32_t e : inside)
        for (int a = 0; a < 3; ++a)
          if (el[e].lo[a] < s.lo[a] || el[e].hi[a] > s.hi[a]) return -2;  // support not a union of elements
      int a = 0;
      for (; a < 3; ++a) {
        traversing_knots(bs[id], inside, a, knots);
        if (!knots.empty()) break;
      }
      if (a == 3) continue;  // minimal support
      const BSpl b = bs[id];
      const int pa = p[a];
      cur.clear();
      Win w0;
      for (int j = 0; j <= pa + 1; ++j) w0.k[j] = kn(b, a, j);
      w0.w = 1.0;
      cur.push_back(w0);
      for (int32_t t : knots) {
        nxt.clear();
        for (const Win& w : cur) {
          bool inner = w.k[0] < t && t < w.k[pa + 1];
          for (int j = 0; j <= pa + 1 && inner; ++j) inner = (w.k[j] != t);
          if (!inner) {
            nxt.push_back(w);
            continue;
          }
          int32_t xn[kMaxP + 3];
          int m = 0;
          bool put = false;
          for (int j = 0; j <= pa + 1; ++j) {
            if (!put && t < w.k[j]) {
              xn[m++] = t;
              put = true;
            }
            xn[m++] = w.k[j];
          }
          double a1 = (t >= w.k[pa]) ? 1.0 : (double)(t - w.k[0]) / (double)(w.k[pa] - w.k[0]);
          double a2 = (t <= w.k[1]) ? 1.0 : (double)(w.k[pa + 1] - t) / (double)(w.k[pa + 1] - w.k[1]);
          for (int c = 0; c < 2; ++c) {
            Win cw;
            for (int j = 0; j <= pa + 1; ++j) cw.k[j] = xn[j + c];
            cw.w = w.w * (c == 0 ? a1 : a2);
            bool merged = false;
            for (Win& o : nxt)
              if (std::equal(o.k, o.k + pa + 2, cw.k)) {
                o.w += cw.w;
                merged = true;
                break;
              }
            if (!merged) nxt.push_back(cw);
          }
        }
        cur.swap(nxt);
      }
      bs[id].alive = false;
      index.erase(b.k);
      for (const Win& w : cur) {
        Key k = b.k;
        for (int j = 0; j <= pa + 1; ++j) k[a * (kMaxP + 2) + j] = w.k[j];
        double g[3] = {w.w * b.gc[0], w.w * b.gc[1], w.w * b.gc[2]};
        size_t before = bs.size();
        int64_t cid = add_bspline(k, w.w * b.gamma, g);
        if (bs.size() != before) {
          heap.push_back({volume(support(bs[cid])), cid});
          std::push_heap(heap.begin(), heap.end());
        }
      }
    }
    return 0;
  }

  int refine(const uint8_t* marked) {
    // B-splines whose support meets a marked element
    std::vector<int32_t> tmp;
    struct Rect {
      int a;
      int32_t t;
      Box r;
    };
    std::vector<Rect> rects;
    for (size_t id = 0; id < bs.size(); ++id) {
      if (!bs[id].alive) continue;
      Box s = support(bs[id]);
      query(s, tmp);
      bool sel = false;
      for (int32_t e : tmp)
        if (marked[e]) {
          sel = true;
          break;
        }
      if (!sel) continue;
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j <= p[a]; ++j) {
          int32_t k0 = kn(bs[id], a, j), k1 = kn(bs[id], a, j + 1);
          if (k0 == k1) continue;
          if ((k0 + k1) & 1) return -3;  // grid too coarse for another halving
          rects.push_back({a, (k0 + k1) / 2, s});
        }
    }
    for (const Rect& r : rects) insert_rectangle(r.a, r.t, r.r);
    int rc = closure();
    compact();
    return rc;
  }

  void compact() {
    std::vector<BSpl> keep;
    keep.reserve(bs.size());
    for (auto& b : bs)
      if (b.alive) keep.push_back(b);
    bs.swap(keep);
    index.clear();
    for (size_t i = 0; i < bs.size(); ++i) index[bs[i].k] = (int64_t)i;
    rebuild_buckets();
  }
};

}  // namespace

extern "C" {

void* lrgen_new(const int* deg, const int* nbase, int levels, int ncomp) {
  for (int a = 0; a < 3; ++a) {
    if (deg[a] < 1 || deg[a] > kMaxP || nbase[a] < 1) return nullptr;
    if ((int64_t)nbase[a] << levels > (1 << 26)) return nullptr;
  }
  if (ncomp < 1 || ncomp > 3) return nullptr;
  Gen* g = new Gen();
  g->init(deg, nbase, levels, ncomp);
  return g;
}

void lrgen_free(void* h) { delete static_cast<Gen*>(h); }

int64_t lrgen_num_elements(void* h) { return (int64_t) static_cast<Gen*>(h)->el.size(); }
int64_t lrgen_num_basis(void* h) { return (int64_t) static_cast<Gen*>(h)->bs.size(); }

// Integer grid resolution per axis (knots and faces are multiples of 1/G_a).
void lrgen_grid(void* h, int* G) {
  Gen* g = static_cast<Gen*>(h);
  for (int a = 0; a < 3; ++a) G[a] = g->G[a];
}

// Element boxes as integers: n_elem x 6 (lo xyz, hi xyz).
void lrgen_elements_int(void* h, int32_t* out) {
  Gen* g = static_cast<Gen*>(h);
  for (size_t e = 0; e < g->el.size(); ++e)
    for (int a = 0; a < 3; ++a) {
      out[e * 6 + a] = g->el[e].lo[a];
      out[e * 6 + 3 + a] = g->el[e].hi[a];
    }
}

// Knots as integers: n_basis x (p0+2 + p1+2 + p2+2), x then y then z.
void lrgen_knots_int(void* h, int32_t* out) {
  Gen* g = static_cast<Gen*>(h);
  int w = g->p[0] + g->p[1] + g->p[2] + 6;
  for (size_t i = 0; i < g->bs.size(); ++i) {
    int m = 0;
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j <= g->p[a] + 1; ++j) out[i * w + m++] = g->kn(g->bs[i], a, j);
  }
}

void lrgen_gamma(void* h, double* out) {
  Gen* g = static_cast<Gen*>(h);
  for (size_t i = 0; i < g->bs.size(); ++i) out[i] = g->bs[i].gamma;
}

// Coefficients carried through refinement (gamma*c accumulated / gamma).
void lrgen_carried_coef(void* h, double* out) {
  Gen* g = static_cast<Gen*>(h);
  for (size_t i = 0; i < g->bs.size(); ++i)
    for (int c = 0; c < g->nc; ++c) out[i * g->nc + c] = g->bs[i].gc[c] / g->bs[i].gamma;
}

// Set coefficients of the current B-splines (n_basis x ncomp); they are then
// carried through later refinements.
void lrgen_set_coef(void* h, const double* coef) {
  Gen* g = static_cast<Gen*>(h);
  for (size_t i = 0; i < g->bs.size(); ++i)
    for (int c = 0; c < g->nc; ++c) g->bs[i].gc[c] = coef[i * g->nc + c] * g->bs[i].gamma;
}

// One structured-mesh refinement pass; marked has one byte per current element.
// Returns 0, or a negative code: -2 broken support invariant, -3 grid too coarse.
int lrgen_refine(void* h, const uint8_t* marked) { return static_cast<Gen*>(h)->refine(marked); }

// n uniforms in [0,1) from std::mt19937_64(seed): (x >> 11) * 2^-53.
void lrgen_uniforms(uint64_t seed, int64_t n, double* out) {
  std::mt19937_64 rng(seed);
  for (int64_t i = 0; i < n; ++i) out[i] = (double)(rng() >> 11) * (1.0 / 9007199254740992.0);
}

}  // extern "C"
