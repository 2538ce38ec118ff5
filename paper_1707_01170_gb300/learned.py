"""Learned step sizes: training on the GPU and per-frame multipliers.

The Eq. 4 step ds(e) of element e is multiplied by m_e = 2^clamp(y_e - margin,
ymin, ymax), with y_e the output of the 16-64-64-64-1 network declared in
lrvol.h, run on the block-local features of e for the frame's camera and
transfer function.  Eq. 4 stays the fallback (every m_e = 1).

Training data come from the renderer itself.  For each seeded training
camera, lrvol_labels marches the Eq. 4 walk and, for every visited element,
finds the largest candidate multiplier whose segment composite stays within
tau of the fine-step (h_fine) composite over the same stretch of ray; the
regression target is log2 of that candidate.  Training runs the library's
FP32 forward / backward kernels and its Adam step; inference runs its BF16
tensor-core kernel.  All arithmetic on the data path happens in the library;
this module only moves tensors and keeps the parameters.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field

import numpy as np

from . import lrvol as lv
from .synth.lrgen import Stream

CAND = (1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0)
# candidates of the refining recipe: also steps below Eq. 4 (m >= 1/2), for
# volumes and transfer functions where Eq. 4 itself is too coarse
CAND_REFINE = (0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0)
MAGIC = b"LRVOLMLP"
FORMAT_VERSION = 2

# parameter layout of lrvol.h: W1[16][64], b1, W2[64][64], b2, W3[64][64], b3, W4[64], b4
_IN, _HID = lv.MLP_IN, lv.MLP_HIDDEN
_LAYERS = [(_IN, _HID), (_HID, _HID), (_HID, _HID), (_HID, 1)]


@dataclass
class TrainConfig:
    seed: int = 1707011790
    h_fine: float = 1.0 / 2048
    tau: float = 4e-4
    cand: tuple = CAND
    steps: int = 2000
    batch: int = 8192
    lr: float = 2e-3
    lr_final: float = 1e-4
    margin: float = 0.25         # subtracted from y at inference (conservative bias)
    ymax: float = 3.0            # log2 of the largest multiplier
    ymin: float = 0.0            # log2 of the smallest multiplier (< 0: steps below Eq. 4)
    extra: dict = field(default_factory=dict)


def refine_config(**kw) -> TrainConfig:
    """The refining recipe: candidates from 1/2 to 8 and multipliers clamped
    to [2^-1, 2^3], so the network can also ask for steps finer than Eq. 4
    where the Eq. 4 step misses the error bar.  The default recipe (steps at
    least Eq. 4's) is faster where Eq. 4 already meets it."""
    return TrainConfig(cand=CAND_REFINE, ymin=-1.0, **kw)


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights from the seeded stream, zero biases (FP32 host array)."""
    u = Stream(seed, lv.MLP_PARAMS + 16).take(lv.MLP_PARAMS)
    p = np.zeros(lv.MLP_PARAMS, dtype=np.float64)
    o = 0
    for fan_in, fan_out in _LAYERS:
        n = fan_in * fan_out
        bound = np.sqrt(6.0 / fan_in)
        p[o:o + n] = bound * (2.0 * u[o:o + n] - 1.0)
        o += n + (fan_out if fan_out > 1 else 1)
    assert o == lv.MLP_PARAMS
    return p.astype(np.float32)


def _bias_out_index() -> int:
    return lv.MLP_PARAMS - 1


class StepModel:
    """Trained parameters (FP32 master copy on the device) and their BF16 packing."""

    def __init__(self, params, cfg: TrainConfig):
        import torch
        self.cfg = cfg
        self.params = torch.as_tensor(np.asarray(params, dtype=np.float32)).cuda().contiguous()
        self._packed = None
        self.train_info = {}

    @property
    def packed(self):
        """BF16 fragments of the parameters with the margin folded into b4."""
        import torch
        if self._packed is None:
            p = self.params.clone()
            p[_bias_out_index()] -= self.cfg.margin
            self._packed = lv.mlp_pack(p)
            torch.cuda.current_stream().synchronize()
        return self._packed

    def multipliers(self, gvol, cam, tf, step, feat=None, out=None, stream=None):
        """Per-element step multipliers for one frame (float32 CUDA tensor, n_elem)."""
        feat = lv.features(gvol, cam, tf, step, out=feat, stream=stream)
        return lv.mlp_infer(feat, self.packed, self.cfg.ymax, out=out, stream=stream, ymin=self.cfg.ymin)

    def save(self, path: str) -> None:
        c = self.cfg
        head = struct.pack("<8sIIddddddI", MAGIC, FORMAT_VERSION, lv.MLP_PARAMS, c.h_fine, c.tau, c.margin, c.ymin,
                           c.ymax, float(c.seed), len(c.cand))
        with open(path, "wb") as f:
            f.write(head)
            f.write(np.asarray(c.cand, dtype="<f4").tobytes())
            f.write(self.params.cpu().numpy().astype("<f4").tobytes())

    @classmethod
    def load(cls, path: str) -> "StepModel":
        with open(path, "rb") as f:
            data = f.read()
        fmt = "<8sIIddddddI"
        n0 = struct.calcsize(fmt)
        magic, ver, npar, h_fine, tau, margin, ymin, ymax, seed, ncand = struct.unpack(fmt, data[:n0])
        if magic != MAGIC or ver != FORMAT_VERSION or npar != lv.MLP_PARAMS:
            raise ValueError(f"{path}: not a step model of format {FORMAT_VERSION} with {lv.MLP_PARAMS} parameters")
        cand = np.frombuffer(data, dtype="<f4", count=ncand, offset=n0)
        params = np.frombuffer(data, dtype="<f4", count=npar, offset=n0 + 4 * ncand)
        cfg = TrainConfig(seed=int(seed), h_fine=h_fine, tau=tau, cand=tuple(float(x) for x in cand), margin=margin,
                          ymin=ymin, ymax=ymax)
        return cls(params.copy(), cfg)


def dataset(gvol, cams, tf, step, cfg: TrainConfig, stream=None):
    """Features and targets log2(cand[label]) of every element visited by each camera.

    Returns (X, target) as CUDA tensors (rows x 16, rows)."""
    import torch
    logc = torch.log2(torch.tensor(cfg.cand, dtype=torch.float32, device="cuda"))
    xs, ts = [], []
    for cam in cams:
        lab = lv.labels(gvol, cam, tf, step, cfg.h_fine, cfg.tau, cfg.cand, stream=stream)
        feat = lv.features(gvol, cam, tf, step, stream=stream)
        sel = lab < len(cfg.cand)
        xs.append(feat[sel])
        ts.append(logc[lab[sel].long()])
    return torch.cat(xs), torch.cat(ts)


def train(X, target, cfg: TrainConfig, log_every: int = 0):
    """Adam on mini-batches drawn from a seeded permutation; returns (model, losses)."""
    import torch
    n = int(X.shape[0])
    if n == 0:
        raise ValueError("empty training set")
    batch = min(cfg.batch, n)
    params = torch.as_tensor(init_params(cfg.seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    scratch = lv.mlp_scratch(batch)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg.seed)
    losses = []
    perm, pos = None, n
    for it in range(1, cfg.steps + 1):
        if pos + batch > n:
            perm, pos = torch.randperm(n, generator=gen, device="cuda"), 0
        idx = perm[pos:pos + batch]
        pos += batch
        # cosine decay from lr to lr_final
        lr = cfg.lr_final + 0.5 * (cfg.lr - cfg.lr_final) * (1 + np.cos(np.pi * (it - 1) / max(1, cfg.steps - 1)))
        lv.mlp_train_step(X[idx].contiguous(), target[idx].contiguous(), params, m, v, it, lr, scratch, loss)
        if log_every and (it == 1 or it % log_every == 0 or it == cfg.steps):
            losses.append((it, float(loss.item())))
    if not losses:
        losses.append((cfg.steps, float(loss.item())))
    return StepModel(params.cpu().numpy(), cfg), losses


def fit(volumes, step, cfg: TrainConfig | None = None, cams_per_volume: int = 32, width: int = 320,
        height: int = 180, log_every: int = 500):
    """The training recipe: labels and features of `cams_per_volume` seeded
    cameras per (volume, transfer function) pair, then Adam.  Volumes must be
    scalar with FP32 storage.  Returns (model, losses, rows)."""
    import torch
    cfg = cfg or TrainConfig()
    Xs, ts = [], []
    for q, (gvol, tf) in enumerate(volumes):
        cams = training_cameras(cfg.seed + 1 + q, cams_per_volume, width, height)
        X, t = dataset(gvol, cams, tf, step, cfg)
        Xs.append(X)
        ts.append(t)
    X, t = torch.cat(Xs), torch.cat(ts)
    model, losses = train(X, t, cfg, log_every=log_every)
    # what a loss near 0.25 means: half the variance of the targets is the
    # loss of the best constant prediction; the labels' own spread (one
    # element, several visits and cameras) puts a floor under any predictor
    model.train_info = {"rows": int(X.shape[0]), "loss_first": losses[0][1], "loss_final": losses[-1][1],
                        "loss_of_best_constant": float(0.5 * torch.var(t, unbiased=False)),
                        "label_histogram": torch.bincount(
                            torch.searchsorted(torch.log2(torch.tensor(cfg.cand, device="cuda")), t),
                            minlength=len(cfg.cand)).tolist()}
    return model, losses, int(X.shape[0])


def training_cameras(seed: int, count: int, width: int, height: int):
    """Seeded perspective orbit cameras (distinct from any evaluation camera)."""
    from .synth.volumes import orbit_camera
    st = Stream(seed, 4 * count + 16)
    return [orbit_camera(st, width, height) for _ in range(count)]


# feature column of the largest TF opacity over the element's value range (lrvol.h)
FEAT_ALPHA_MAX = 6


def rule_multipliers(feat, theta: float, big: float, small: float):
    """A one-line per-element rule on the features the network sees: the
    multiplier `big` where the largest TF opacity over the element's value
    range is at most theta (the element is (nearly) empty for this TF), else
    `small`.  A baseline for the network, not used by the renderer."""
    import torch
    return torch.where(feat[:, FEAT_ALPHA_MAX] <= theta, big, small).to(torch.float32).contiguous()


def ablation(gvol, cam, tf, step, model, fine, target: float = 1e-3, stream=None):
    """Samples (as a fraction of Eq. 4's) and image RMSE against the fine-step
    reference `fine` for: Eq. 4; every constant multiplier of the candidate
    set; the empty-element rule (8x where the TF's largest opacity over the
    element's range is 0, else 1x) and its tuned family (threshold theta,
    multiplier c elsewhere); and the trained network.  For each family the
    best member is the one with the fewest samples at RMSE <= target, and,
    separately, at RMSE <= the network's own RMSE."""
    import torch
    from .synth.volumes import StepParams

    def run(mult):
        s = StepParams(mode="learned", xi=step.xi, alpha_stop=step.alpha_stop, field=step.field,
                       component=step.component, mult=mult)
        img = gvol.render(cam, tf, s, stream=stream)
        n = gvol.stats()["samples"]
        return n, float(torch.sqrt(torch.mean((img.double() - fine.double()) ** 2)))

    heur = gvol.render(cam, tf, step, stream=stream)
    n0 = gvol.stats()["samples"]
    e0 = float(torch.sqrt(torch.mean((heur.double() - fine.double()) ** 2)))
    feat = lv.features(gvol, cam, tf, step, stream=stream)
    nel = feat.shape[0]
    rows = {"eq4": (1.0, e0)}
    consts = {}
    for c in model.cfg.cand:
        n, e = run(torch.full((nel,), float(c), dtype=torch.float32, device="cuda"))
        consts[c] = (n / n0, e)
    rules = {}
    for theta in (0.0, 1e-3, 3e-3, 1e-2):
        for c in model.cfg.cand[:4]:
            n, e = run(rule_multipliers(feat, theta, float(max(model.cfg.cand)), float(c)))
            rules[(theta, c)] = (n / n0, e)
    n, e = run(model.multipliers(gvol, cam, tf, step, stream=stream))
    rows["network"] = (n / n0, e)
    rows["rule_empty_8x_else_1x"] = rules[(0.0, model.cfg.cand[0])]

    def best(table, bar):
        ok = [(v[0], k, v[1]) for k, v in table.items() if v[1] <= bar]
        if not ok:
            return None
        f, k, e = min(ok)
        return {"param": k, "samples_frac": f, "rmse": e}

    e_net = rows["network"][1]
    return {
        "target_rmse": target, "eq4_samples": n0, "eq4_rmse": e0,
        "network": {"samples_frac": rows["network"][0], "rmse": e_net},
        "rule_empty_8x_else_1x": {"samples_frac": rows["rule_empty_8x_else_1x"][0],
                                  "rmse": rows["rule_empty_8x_else_1x"][1]},
        "best_constant_at_target": best(consts, target),
        "best_constant_at_network_rmse": best(consts, e_net),
        "best_rule_at_target": best(rules, target),
        "best_rule_at_network_rmse": best(rules, e_net),
        "constants": {str(k): {"samples_frac": v[0], "rmse": v[1]} for k, v in consts.items()},
        "rules": {f"theta={k[0]:g},else={k[1]:g}": {"samples_frac": v[0], "rmse": v[1]} for k, v in rules.items()},
    }
