"""FP64 oracle of the density control the mapper runs between optimisation
steps -- test infrastructure only.

The paper keeps the map covering the scene by adaptive density control: the
3DGS strategy that clones and splits Gaussians from their size and view-space
gradient, or the MCMC strategy that relocates low-opacity Gaussians and adds
noise, with an upper bound on their number and lr_noise = 1e4 (Sec. 3.3, last
paragraph; Supp. "Monte Carlo Markov Chain Gaussian Splatting").  It cites
both methods without restating them; these are restatements of the published
steps, with the readings below.

Adaptive density control (3DGS), one pass over Gaussians g = 0..N-1:
  mean gradient  g_bar = grad_g / count_g (0 without views)
  dense          g_bar >= grad_threshold
  big            max_k s_gk > split_scale          (s = exp(log-scales))
  pruned         sigma_g < min_opacity, or radius_g > max_screen_radius (if
                 that is > 0), or max_k s_gk > max_world_scale (if > 0)
  output, in g order: nothing if pruned; else two children if dense and big
  (mean mu + R diag(s) eps_c for the two given standard-normal draws eps_c,
  log-scales - ln 1.6, the rest copied); else the Gaussian and, if dense, an
  exact copy.  Every decision is taken on the Gaussian as it came in.
  Decisions compare exactly: grad >= threshold * count in FP64 (both factors
  FP32, so the product is exact), log-scales against ln(threshold) in FP64,
  logits against logit(min_opacity) in FP64.

MCMC relocation (3DGS-MCMC), Gaussians "dead" at opacity <= min_opacity:
  each dead slot d draws a live source s_d with probability proportional to
  its opacity, by the inverse CDF of integer weights w_g = floor(o32_g 2^24)
  at t_d = floor(r_d W / 2^32) (W = sum of weights, r_d the slot's uniform
  32-bit draw): s_d = the first g whose inclusive weight sum exceeds t_d.
  o32 is the FP32 sigmoid of sigmoid32 below, taken identically by the
  kernel, so both sides make the same integer choices.  A source drawn n
  times ends with k = n + 1 identical Gaussians: each with opacity
  o' = 1 - (1 - o)^(1/k) (so that k stacked copies have opacity o) and scales
  multiplied by
      c = o / sum_{i=1..k} sum_{j=0..i-1} C(i-1, j) (-1)^j o'^(j+1) / sqrt(j+1),
  which keeps the integral of the composited opacity profile; o' is clamped
  to [min_opacity, 1 - 2^-23] so that the logit stays finite, and k is capped
  at MAX_COPIES = 51 in both formulas (the published rule's table size; the
  alternating binomial sum loses all precision far beyond it).  With no live
  Gaussian nothing moves.

MCMC noise (3DGS-MCMC):
  mu += scale sigma(-100 (o - 0.005)) Sigma eta,  Sigma = R diag(s^2) R^T,
  eta the given standard-normal draw; scale = lr_noise x the position
  learning rate.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Tuple

import numpy as np

SPLIT_FACTOR = 1.6
NOISE_K = 100.0
NOISE_T = 0.005
WEIGHT_BITS = 24
MAX_COPIES = 51
_F = np.float32


# ---------------------------------------------------------------- FP32 sigmoid for the sampling weights
# exp by Cody-Waite range reduction (x = n ln2 + f, |f| <= ln2 / 2, ln 2 split
# into an exactly representable high part and a low part) and the degree-7
# Taylor polynomial of e^f in Horner form, then scaling by 2^n.  Every step is
# one correctly rounded FP32 operation, so any IEEE implementation of the same
# sequence gives the same bits.
LN2_HI = _F(0.693145751953125)          # 15 significant bits: n * LN2_HI is exact for |n| < 2^9
LN2_LO = _F(math.log(2.0) - 0.693145751953125)
LOG2E = _F(1.0 / math.log(2.0))
EXP_COEF = [_F(1.0 / math.factorial(k)) for k in range(8)]


def exp32(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=_F)
    x = np.clip(x, _F(-87.0), _F(88.0))
    n = np.rint(x * LOG2E).astype(_F)
    f = (x - n * LN2_HI) - n * LN2_LO
    p = EXP_COEF[7]
    for k in range(6, -1, -1):
        p = p * f + EXP_COEF[k]
    return np.ldexp(p, n.astype(np.int32)).astype(_F)


def sigmoid32(logit: np.ndarray) -> np.ndarray:
    one = _F(1.0)
    return (one / (one + exp32(-np.asarray(logit, dtype=_F)))).astype(_F)


def weights(logit: np.ndarray, min_opacity: float) -> Tuple[np.ndarray, np.ndarray]:
    """(dead mask, integer sampling weights) of the MCMC relocation."""
    o32 = sigmoid32(logit)
    dead = o32 <= _F(min_opacity)
    w = np.floor(o32.astype(np.float64) * (1 << WEIGHT_BITS)).astype(np.int64)
    w[dead] = 0
    return dead, w


# ---------------------------------------------------------------- shared helpers
def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """[4][N] (w, x, y, z), unnormalised -> [N][3][3]."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=0, keepdims=True)
    w, x, y, z = q
    R = np.empty((q.shape[1], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def logit(p):
    p = np.asarray(p, np.float64)
    return np.log(p / (1.0 - p))


@dataclass
class Gaussians:
    """Planar parameters, like the kernel's: means [3][N], log_scales [3][N],
    quats [4][N], opacity_logits [N], sh [C][N]."""
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray

    @property
    def N(self) -> int:
        return int(self.opacity_logits.shape[0])

    def take(self, idx) -> "Gaussians":
        idx = np.asarray(idx, np.int64)
        return Gaussians(self.means[:, idx].copy(), self.log_scales[:, idx].copy(), self.quats[:, idx].copy(),
                         self.opacity_logits[idx].copy(), self.sh[:, idx].copy())

    def as64(self) -> "Gaussians":
        return Gaussians(*(np.asarray(a, np.float64) for a in
                           (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)))


# ---------------------------------------------------------------- adaptive density control
def adc_decisions(g: Gaussians, grad, count, radius, grad_threshold, split_scale, min_opacity,
                  max_screen_radius=0.0, max_world_scale=0.0) -> Dict[str, np.ndarray]:
    # thresholds arrive as FP32 (the C ABI's type)
    split_scale, min_opacity = float(_F(split_scale)), float(_F(min_opacity))
    max_screen_radius, max_world_scale = float(_F(max_screen_radius)), float(_F(max_world_scale))
    ls_max = np.max(np.asarray(g.log_scales, np.float64), axis=0)
    grad = np.asarray(grad, np.float32).astype(np.float64)
    count = np.asarray(count, np.float32).astype(np.float64)
    dense = (count > 0) & (grad >= float(np.float32(grad_threshold)) * count)
    big = ls_max > math.log(split_scale)
    pruned = np.asarray(g.opacity_logits, np.float64) < math.log(min_opacity / (1.0 - min_opacity))
    if max_screen_radius > 0:
        pruned |= np.asarray(radius, np.float32) > np.float32(max_screen_radius)
    if max_world_scale > 0:
        pruned |= ls_max > math.log(max_world_scale)
    split = dense & big & ~pruned
    clone = dense & ~big & ~pruned
    n_out = np.where(pruned, 0, np.where(split | clone, 2, 1))
    return dict(dense=dense, big=big, pruned=pruned, split=split, clone=clone, n_out=n_out)


def adc(g: Gaussians, grad, count, radius, normals, grad_threshold, split_scale, min_opacity,
        max_screen_radius=0.0, max_world_scale=0.0) -> Gaussians:
    """normals: [2][3][N] standard-normal draws for the split children."""
    d = adc_decisions(g, grad, count, radius, grad_threshold, split_scale, min_opacity, max_screen_radius,
                      max_world_scale)
    g64 = g.as64()
    R = quat_to_rot(g64.quats)
    s = np.exp(g64.log_scales)                       # [3][N]
    normals = np.asarray(normals, np.float64)
    cols = {k: [] for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    for i in range(g.N):   # one Gaussian at a time, in order
        if d["pruned"][i]:
            continue
        if d["split"][i]:
            for c in range(2):
                offset = R[i] @ (s[:, i] * normals[c, :, i])
                cols["means"].append(g64.means[:, i] + offset)
                cols["log_scales"].append(g64.log_scales[:, i] - math.log(SPLIT_FACTOR))
                cols["quats"].append(g64.quats[:, i])
                cols["opacity_logits"].append(g64.opacity_logits[i])
                cols["sh"].append(g64.sh[:, i])
            continue
        copies = 2 if d["clone"][i] else 1
        for _ in range(copies):
            cols["means"].append(g64.means[:, i])
            cols["log_scales"].append(g64.log_scales[:, i])
            cols["quats"].append(g64.quats[:, i])
            cols["opacity_logits"].append(g64.opacity_logits[i])
            cols["sh"].append(g64.sh[:, i])
    if not cols["means"]:
        return Gaussians(np.zeros((3, 0)), np.zeros((3, 0)), np.zeros((4, 0)), np.zeros(0),
                         np.zeros((g.sh.shape[0], 0)))
    return Gaussians(np.stack(cols["means"], 1), np.stack(cols["log_scales"], 1), np.stack(cols["quats"], 1),
                     np.array(cols["opacity_logits"]), np.stack(cols["sh"], 1))


# ---------------------------------------------------------------- MCMC relocation
def relocation_opacity(o, k):
    """Opacity of each of k stacked copies that together have opacity o."""
    return 1.0 - (1.0 - np.asarray(o, np.float64)) ** (1.0 / np.asarray(k, np.float64))


def relocation_scale_factor(o, o_new, k: int) -> float:
    """The double sum of the relocation rule, term by term."""
    den = 0.0
    for i in range(1, k + 1):
        for j in range(i):
            den += math.comb(i - 1, j) * (-1) ** j * o_new ** (j + 1) / math.sqrt(j + 1)
    return o / den


def relocate_sources(logit_, r, min_opacity):
    """(dead mask, source of every dead slot (-1 elsewhere), times each
    Gaussian was drawn) for uniform 32-bit draws r[N]."""
    dead, w = weights(logit_, min_opacity)
    N = len(w)
    src = np.full(N, -1, np.int64)
    drawn = np.zeros(N, np.int64)
    W = int(w.sum())
    if W == 0:
        return dead, src, drawn
    cum = np.cumsum(w)
    for d in np.nonzero(dead)[0]:
        t = (int(r[d]) * W) >> 32
        s = int(np.searchsorted(cum, t, side="right"))   # first g with cum[g] > t
        src[d] = s
        drawn[s] += 1
    return dead, src, drawn


def mcmc_relocate(g: Gaussians, r, min_opacity: float) -> Tuple[Gaussians, np.ndarray]:
    """Returns (the relocated Gaussians, the source of every dead slot)."""
    min_opacity = float(_F(min_opacity))
    dead, src, drawn = relocate_sources(g.opacity_logits, r, min_opacity)
    out = g.as64()
    new = g.as64()
    o = sigmoid(new.opacity_logits)
    for s in np.nonzero(drawn)[0]:
        k = min(int(drawn[s]) + 1, MAX_COPIES)
        o_new = float(relocation_opacity(o[s], k))
        o_new = min(max(o_new, min_opacity), 1.0 - 2.0 ** -23)
        c = relocation_scale_factor(o[s], o_new, k)
        new.opacity_logits[s] = logit(o_new)
        new.log_scales[:, s] = new.log_scales[:, s] + math.log(c)
    for i in range(g.N):
        j = src[i] if src[i] >= 0 else i
        out.means[:, i] = new.means[:, j]
        out.log_scales[:, i] = new.log_scales[:, j]
        out.quats[:, i] = new.quats[:, j]
        out.opacity_logits[i] = new.opacity_logits[j]
        out.sh[:, i] = new.sh[:, j]
    return out, src


# ---------------------------------------------------------------- MCMC noise
def mcmc_noise(g: Gaussians, eta, scale: float) -> np.ndarray:
    """New means [3][N] for the standard-normal draws eta [3][N]."""
    g64 = g.as64()
    R = quat_to_rot(g64.quats)
    s2 = np.exp(2.0 * g64.log_scales)
    Sigma = np.einsum("nij,jn,nkj->nik", R, s2, R)
    o = sigmoid(g64.opacity_logits)
    gate = sigmoid(-NOISE_K * (o - NOISE_T))
    step = np.einsum("nij,jn->in", Sigma, np.asarray(eta, np.float64))
    return g64.means + scale * gate[None, :] * step
