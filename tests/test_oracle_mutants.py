"""Planted mistakes: every plausible slip in the oracle must trip a pin.

Each case edits one line of oracle.c (a dropped term, a wrong index or sign,
a transposed axis, an off-by-one), builds the edited copy on the CPU into a
temporary directory, points the oracle module at it, and runs the pins of
test_oracle_pins, the label pins of test_oracle_learned and the gradient and
shading pins of test_oracle_shading, the streamline pins of
test_oracle_streamlines, the trimming pins of test_oracle_trim and the
per-sample trace pins of test_oracle_trace; at least
one must fail.  The default build is restored
afterwards.  No GPU is involved.
"""
import os
import pytest

import oracle.oracle as orc

import test_oracle_learned as L
import test_oracle_shading as S
import test_oracle_streamlines as SL
import test_oracle_trim as T
import test_oracle_tubes as TU
import test_oracle_pins as P
import test_oracle_trace as TR

SRC = os.path.join(os.path.dirname(orc.__file__), "oracle.c")

MUTANTS = [
    ("Cox-de Boor drops the right term", "N[j] = left + right;", "N[j] = left;"),
    ("Cox-de Boor right term uses a wrong knot",
     "right = (xi[j + r + 1] - x) / (xi[j + r + 1] - xi[j + 1]) * N[j + 1];",
     "right = (xi[j + r] - x) / (xi[j + r + 1] - xi[j + 1]) * N[j + 1];"),
    ("Cox-de Boor starts from closed intervals", "N[j] = (xi[j] <= x && x < xi[j + 1]) ? 1.0 : 0.0;",
     "N[j] = (xi[j] <= x && x <= xi[j + 1]) ? 1.0 : 0.0;"),
    ("Eq. 2 without the scale factors gamma", "double N = v->weight[i];", "double N = 1.0;"),
    ("Eq. 2 evaluates every factor on the x knots",
     "for (int a = 0; a < 3; ++a) N *= orc_bspline(knots_of(v, i, a), v->p[a], x[a]);",
     "for (int a = 0; a < 3; ++a) N *= orc_bspline(knots_of(v, i, 0), v->p[a], x[a]);"),
    ("Eq. 2 evaluates a factor at the wrong coordinate",
     "for (int a = 0; a < 3; ++a) N *= orc_bspline(knots_of(v, i, a), v->p[a], x[a]);",
     "for (int a = 0; a < 3; ++a) N *= orc_bspline(knots_of(v, i, a), v->p[a], x[(a + 1) % 3]);"),
    ("incidence misses supports that start at the element",
     "ok = (k[0] <= b[a]) && (b[3 + a] <= k[v->p[a] + 1]);",
     "ok = (k[0] < b[a]) && (b[3 + a] <= k[v->p[a] + 1]);"),
    ("element boxes closed at the top", "if (!(lo <= x[a] && (x[a] < hi || (x[a] == hi && hi == 1.0)))) return 0;",
     "if (!(lo <= x[a] && (x[a] <= hi))) return 0;"),
    ("Alg. 2 drops the (1 - alpha_dst) factor", "double w = (1.0 - T) * (1.0 - A);", "double w = (1.0 - T);"),
    ("Alg. 2 ignores the segment length", "double T = pow(1.0 - src[3], seg / J->st->xi);",
     "double T = 1.0 - src[3];"),
    ("segment not clipped at the exit", "double seg = (double)fminf(tn, tout) - (double)t;",
     "double seg = (double)tn - (double)t;"),
    ("Eq. 4 with 2^-(d-1)", "return (float)ldexp(m, -d);", "return (float)ldexp(m, -d + 1);"),
    ("Eq. 4 with the longest side", "if (b[4] - b[1] < m) m = b[4] - b[1];", "if (b[4] - b[1] > m) m = b[4] - b[1];"),
    ("TF weights swapped",
     "rgba[c] = (1.0 - f) * tf->table[4 * i0 + c] + f * tf->table[4 * (i0 + 1) + c];",
     "rgba[c] = f * tf->table[4 * i0 + c] + (1.0 - f) * tf->table[4 * (i0 + 1) + c];"),
    ("image rows flipped", "k->sys = (float)(-2.0 * ty / (double)c->height);",
     "k->sys = (float)(2.0 * ty / (double)c->height);"),
    ("camera right vector sign", "R[0] = F[1] * c->up[2] - F[2] * c->up[1];",
     "R[0] = F[2] * c->up[1] - F[1] * c->up[2];"),
    ("slab test uses the wrong face", "float tb = (1.0f - o[c]) * inv;", "float tb = (0.5f - o[c]) * inv;"),
    ("fixed step doubled", "tn = fmaf((float)(k + 1), (float)J->st->h, tin);",
     "tn = fmaf((float)(k + 1), 2.0f * (float)J->st->h, tin);"),
    ("learned step ignores the multiplier", "tn = t + orc_heuristic_step(v, cur) * J->st->mult[cur];",
     "tn = t + orc_heuristic_step(v, cur);"),
    ("labels judged only over the Eq. 4 visit",
     "seg_composite(v, J->tf, J->st, o, d, t, tc, (float)J->h_fine, &sc, F, &FA);\n"
     "        seg_composite(v, J->tf, J->st, o, d, t, tc, s, &sc, Cc, &CA);",
     "seg_composite(v, J->tf, J->st, o, d, t, tb, (float)J->h_fine, &sc, F, &FA);\n"
     "        seg_composite(v, J->tf, J->st, o, d, t, tb, s, &sc, Cc, &CA);"),
    ("labels ignore the front transmittance", "if (!(Tfront * err <= J->tau)) break;",
     "if (!(err <= J->tau)) break;"),
    ("labels compare candidates with the Eq. 4 step", "float s = ds * J->cand[c], tc = t;",
     "float s = ds, tc = t;"),
    ("B-spline derivative without the factor p", "return (double)p * d;", "return d;"),
    ("B-spline derivative adds the right term",
     "if (xi[p + 1] != xi[1]) d -= orc_bspline(xi + 1, p - 1, x) / (xi[p + 1] - xi[1]);",
     "if (xi[p + 1] != xi[1]) d += orc_bspline(xi + 1, p - 1, x) / (xi[p + 1] - xi[1]);"),
    ("gradient differentiates y for x", "{g * D[0] * B[1] * B[2],", "{g * B[0] * D[1] * B[2],"),
    ("shading ignores the light vector", "l[c] = J->st->light[c];", "l[c] = 0.0;"),
    ("shading without the 0.4 floor", "if (shade < 0.4) shade = 0.4;", ""),
    ("RK4 weight 1/6 for the second stage",
     "T->b[0] = 1.0 / 6; T->b[1] = 1.0 / 3; T->b[2] = 1.0 / 3; T->b[3] = 1.0 / 6;",
     "T->b[0] = 1.0 / 6; T->b[1] = 1.0 / 6; T->b[2] = 1.0 / 3; T->b[3] = 1.0 / 6;"),
    ("Kutta's method with a31 = +1", "T->a[1][0] = 0.5; T->a[2][0] = -1.0; T->a[2][1] = 2.0;",
     "T->a[1][0] = 0.5; T->a[2][0] = 1.0; T->a[2][1] = 2.0;"),
    ("3/8 rule with a42 = +1", "T->a[3][0] = 1.0; T->a[3][1] = -1.0; T->a[3][2] = 1.0;",
     "T->a[3][0] = 1.0; T->a[3][1] = 1.0; T->a[3][2] = 1.0;"),
    ("Fehlberg fifth-order weight sign", "T->b[4] = -9.0 / 50;", "T->b[4] = 9.0 / 50;"),
    ("stages evaluated at x_n", "y[a] = x[a] + hs * acc;", "y[a] = x[a];"),
    ("trimming takes back faces for front faces", "*front = det > 0.0f;", "*front = det < 0.0f;"),
    ("trimming ignores the back faces", "if (tb != 0.0f && tb < *tout) *tout = tb;", ""),
    ("tubes keep the farthest hit", "if (t < tbest) { /* strictly smaller", "if (tbest == INFINITY || t > tbest) { /* strictly smaller"),
    ("tubes without caps", "const float h = bb * bb - cc;", "const float h = -1.0f;"),
    ("tube shading without the 0.4 floor", "if (I < 0.4) I = 0.4;", ""),
    ("streamline Eq. 4 step without the element", "if (P->step_rule == 1) h = P->h * (double)orc_heuristic_step(v, e);",
     "if (P->step_rule == 1) h = P->h;"),
    ("trace keeps the next sample's t", "rec[0] = (double)t;", "rec[0] = (double)tn;"),
    ("trace keeps the unclipped segment", "rec[3] = seg;", "rec[3] = (double)tn - (double)t;"),
    ("trace counts one sample too many", "if (J->count) J->count[q] = (int32_t)k;",
     "if (J->count) J->count[q] = (int32_t)k + 1;"),
]


def _pins(cfg1):
    """The pins of test_oracle_pins, run against whatever library is loaded."""
    O = orc.Oracle(cfg1)
    yield lambda: P.test_bspline_golden_closed_forms()
    yield lambda: P.test_bspline_half_open_support()
    yield lambda: P.test_partition_of_unity((2, 2, 2), (3, 3, 3), (0.4, 0.2), (0.3, 0.6, 0.45))
    yield lambda: P.test_polynomial_reproduction((2, 2, 2), ([0.1, -1.0, 2.0], [0.2, 0.5, -0.3], [1.0, 0.0, 1.0]),
                                                 "carried")
    yield lambda: P.test_tensor_product_special_case()
    yield lambda: P.test_lookup_tiny_partition()
    yield lambda: P.test_bezier_blocks_equal_bspline_evaluation(cfg1, O)
    for which in ("ortho_z", "oblique", "persp"):
        yield lambda which=which: P.test_ray_setup_matches_double(which)
    yield lambda: P.test_ray_ortho_z_exact()
    for mode in ("fixed", "heuristic"):
        for which in ("ortho_z", "persp"):
            yield lambda mode=mode, which=which: P.test_closed_form_opacity(cfg1, mode, which)
    yield lambda: P.test_tf_linear_interpolation(cfg1)
    yield lambda: P.heuristic_count_pin(cfg1, O)
    yield lambda: P.test_heuristic_step_counts_anisotropic()
    yield lambda: P.test_learned_step_counts()
    yield lambda: P.test_early_termination_and_miss(O)
    yield lambda: TR.test_trace_cfg1_oblique(cfg1, O, "heuristic")
    yield lambda: TR.test_trace_matches_render_and_counts(cfg1, O)
    yield lambda: L.test_labels_constant_field_accept_every_candidate(cfg1)
    yield lambda: L.test_labels_monotone_in_tau(cfg1, O)
    yield lambda: L.test_labels_count_what_the_last_step_skips()
    yield lambda: L.test_labels_weigh_errors_by_front_transmittance()
    yield lambda: S.test_bspline_derivative_matches_scipy()
    yield lambda: S.test_gradient_of_reproduced_polynomials((2, 2, 2), ([0.1, -1.0, 2.0], [0.2, 0.5, -0.3],
                                                                        [1.0, 0.0, 1.0]))
    yield lambda: S.test_shading_of_a_constant_field_is_0p4(cfg1)
    yield lambda: S.test_shading_closed_forms_linear_field()
    yield lambda: T.test_box_intervals_along_z()
    yield lambda: T.test_sphere_is_watertight()
    yield lambda: T.test_trimmed_constant_field_closed_form(cfg1, "outside")
    yield lambda: T.test_trimmed_constant_field_closed_form(cfg1, "inside")
    yield lambda: TU.test_straight_segment_closed_form()
    yield lambda: TU.test_caps_and_occlusion()
    H = orc.Oracle(SL.helix_volume())
    for m in sorted(SL.ORDERS):
        yield lambda m=m: SL.test_fixed_step_order(H, m)
    yield lambda: SL.test_constant_field_is_exact_and_heuristic_step_closed_form("RK4")
    yield lambda: SL.test_domain_exit_and_sample_cap()
    for m in ("HE", "BS", "RKF45"):
        yield lambda m=m: SL.test_adaptive_meets_tolerance(H, m)


def test_unmutated_source_passes_the_same_pins(cfg1):
    for pin in _pins(cfg1):
        pin()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path, cfg1):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    msrc = tmp_path / "oracle_mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = orc.build(force=True, src=str(msrc), lib=str(tmp_path / "liboracle_mutant.so"))
    prev = orc.use_library(lib)
    caught = None
    try:
        for pin in _pins(cfg1):
            try:
                pin()
            except (AssertionError, StopIteration, ValueError, IndexError) as exc:
                caught = exc
                break
    finally:
        orc.use_library(prev)
    assert caught is not None, f"no pin caught: {name}"
