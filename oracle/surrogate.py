"""FP64 CPU oracle of the learned echo surrogate (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's oracle legs may import this module.
It imports nothing from the CUDA product package.

The paper (Sec. II.B) proposes learned scattering functions as a way to stand in for
the costly physics of echo formation. The surrogate built here is a small per-beam 1-D
convolutional network that maps a cheap geometric rendering of each beam to the
coherent envelope profile the plain method forms. The paper gives neither the network
nor its inputs; the readings below are this build's, stated next to each function.

Geometric rendering (reading). For every beam one ray leaves along the beam centre
u_b and follows the plain method's isovelocity route rules (mirror reflections at
mirror-flagged facets and at the sea surface, at most max_bounces, stopping past the
one-way length limit). Its first two scatter hits (triangle hits) give per beam
(L_h, kappa_h, mu_h, Gamma_h), h = 1, 2: one-way route length, incidence cosine
|d . n|, facet reflectivity and the route's one-way reflection product; absent hits
are zeros. The ray grid of the plain method with one ray per beam cell and one
sub-ray is exactly this set of rays, so the oracle reads the rendering off its own
route tracer (orc_trace).

Rasterisation (reading). On the range axis (bin centres r_n = r_min + (n + 1/2) dr)
a hit at one-way length L sits at bin coordinate x = (L - r_min) / dr - 1/2 and is
splatted linearly onto bins floor(x) and floor(x) + 1 with weights 1 - f and f
(f = x - floor(x)); bins outside [0, n_range) are dropped. Four input channels:
0 the first hit's splat, 1 the second hit's splat, 2 the incidence cosines and 3 the
reflectivities of both hits, each as the amplitude of its hit's splat.

Network (the configuration's stated shape). Six 1-D convolutions along range, kernel
9, zero padding at both ends of the beam ("same" length), channels
4 -> 64 -> 64 -> 64 -> 64 -> 64 -> 1, ReLU after the first five, linear output. Layer
l computes z[n, o] = b[o] + sum_{c, k} W[o, c, k] x[n + k - 4, c]. The output
yhat[n] approximates E[n] / E_scale, E the plain method's envelope.

Training (reading). Mean-squared error over every (beam, bin) of a batch; Adam
(Kingma & Ba 2015) with bias correction. With bf16=True the oracle rounds to BF16 at
the points where the GPU kernels store BF16 (the activations a_1..a_5 between layers
and the back-propagated dz_1..dz_5), so that the two agree to accumulation order.
"""
from __future__ import annotations

import math

import numpy as np

from . import trace as _trace, pulse_acf as _pulse_acf

KERNEL = 9
HALF = KERNEL // 2
CHANNELS = (4, 64, 64, 64, 64, 64, 1)


# ------------------------------------------------------------------ rendering
def render(scene, params: dict, pose: dict, ssp: dict, use_bvh: bool = True, with_ties: bool = False):
    """Per-beam geometric rendering [n_beam_el * n_beam_az, 8] float64: (L, kappa, mu,
    Gamma) of the first and of the second scatter hit of the beam-centre route; zeros
    where a hit is absent. Isovelocity profiles only. with_ties: also return a [beams]
    bool array, True where every recorded hit of the beam clears the near-tie margins
    (barycentric margin > 1e-5 and distance gap to the runner-up > 1e-6 m)."""
    nb = params["n_beam_az"] * params["n_beam_el"]
    q = dict(params, n_ray_az=params["n_beam_az"], n_ray_el=params["n_beam_el"], n_sub=1, cross=0,
             vol_n=0)
    q.pop("field", None)
    empty = type(scene)(scene.verts, scene.tris, scene.mu, scene.flags)  # mesh only: no point scatterers
    h = _trace(empty, q, pose, ssp, use_bvh=use_bvh)
    out = np.zeros((nb, 8))
    mesh = h["prim"] >= 0
    ray, seg, L = h["ray"][mesh], h["seg"][mesh], h["len"][mesh]
    mu = np.asarray(scene.mu, np.float64)[h["prim"][mesh]]
    kinc, gam = h["kinc"][mesh], h["gam"][mesh]
    tie_free = (h["margin"][mesh] > 1e-5) & (h["gap"][mesh] > 1e-6)
    clear = np.ones(nb, bool)
    # a route's scatter hits in route order: by one-way length
    order = np.lexsort((L, ray))
    seen = {}
    for i in order:
        b = int(ray[i])
        k = seen.get(b, 0)
        if k < 2:
            out[b, 4 * k:4 * k + 4] = (L[i], kinc[i], mu[i], gam[i])
            seen[b] = k + 1
            clear[b] &= bool(tie_free[i])
    return (out, clear) if with_ties else out


def rasterize(feat: np.ndarray, params: dict) -> np.ndarray:
    """Input channels [beams, n_range, 4] from the rendering (linear splats)."""
    nb, nr = feat.shape[0], params["n_range"]
    dr = (params["r_max"] - params["r_min"]) / nr
    X = np.zeros((nb, nr, 4))
    for b in range(nb):
        for h in range(2):
            L, kap, mu, _ = feat[b, 4 * h:4 * h + 4]
            if L <= 0:
                continue
            x = (L - params["r_min"]) / dr - 0.5
            n0 = math.floor(x)
            f = x - n0
            for n, w in ((n0, 1.0 - f), (n0 + 1, f)):
                if 0 <= n < nr:
                    X[b, n, h] += w
                    X[b, n, 2] += kap * w
                    X[b, n, 3] += mu * w
    return X


def geometric_envelope(feat: np.ndarray, params: dict, c_ref: float) -> np.ndarray:
    """The rendering turned into an envelope without the network (the method without
    it): each rendered hit contributes its Lambertian amplitude
    Gamma^2 sqrt(mu kappa dOmega_b) / L exp(-2 alpha L), dOmega_b the beam cell's solid
    angle, shaped by the pulse autocorrelation |R(t_n - 2 L / c)| and the TVG gain;
    contributions add in amplitude. [beams, n_range]."""
    nba, nbe, nr = params["n_beam_az"], params["n_beam_el"], params["n_range"]
    dr = (params["r_max"] - params["r_min"]) / nr
    daz, dele = params["hfov"] / nba, params["vfov"] / nbe
    r = params["r_min"] + (np.arange(nr) + 0.5) * dr
    t = 2.0 * r / c_ref
    tvg = r * np.exp(2.0 * params["alpha"] * r)
    E = np.zeros((feat.shape[0], nr))
    for b in range(feat.shape[0]):
        j = b // nba
        el_lo = -params["vfov"] / 2 + j * dele
        domega = daz * (math.sin(el_lo + dele) - math.sin(el_lo))
        for h in range(2):
            L, kap, mu, gam = feat[b, 4 * h:4 * h + 4]
            if L <= 0:
                continue
            a = gam * gam * math.sqrt(mu * kap * domega) / L * math.exp(-2.0 * params["alpha"] * L)
            tau = 2.0 * L / c_ref
            near = np.nonzero(np.abs(t - tau) < params["pulse"])[0]
            if len(near):
                E[b, near] += a * np.abs(_pulse_acf(t[near] - tau, params["pulse"], params["bw"]))
    return E * tvg


# ------------------------------------------------------------------ network
def bf16(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (round to nearest even from the FP32 rounding of x), as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv(x: np.ndarray, W: np.ndarray, b) -> np.ndarray:
    """z[beam, n, o] = b[o] + sum_{c, k} W[o, c, k] x[beam, n + k - 4, c], x zero outside
    the beam's bins."""
    nb, nr, _ = x.shape
    xp = np.zeros((nb, nr + 2 * HALF, x.shape[2]))
    xp[:, HALF:HALF + nr] = x
    z = np.zeros((nb, nr, W.shape[0]))
    for k in range(KERNEL):
        z += np.einsum("bnc,oc->bno", xp[:, k:k + nr], W[:, :, k])
    if b is not None:
        z += np.asarray(b)[None, None, :]
    return z


def conv_input_grad(dz: np.ndarray, W: np.ndarray) -> np.ndarray:
    """dx[beam, m, c] = sum_{o, k} W[o, c, k] dz[beam, m - k + 4, o] (the adjoint of conv)."""
    nb, nr, _ = dz.shape
    dzp = np.zeros((nb, nr + 2 * HALF, dz.shape[2]))
    dzp[:, HALF:HALF + nr] = dz
    dx = np.zeros((nb, nr, W.shape[1]))
    for k in range(KERNEL):
        # m - k + 4 = (m + (8 - k)) - 4: the padded index m + 8 - k
        dx += np.einsum("bno,oc->bnc", dzp[:, KERNEL - 1 - k:KERNEL - 1 - k + nr], W[:, :, k])
    return dx


def conv_weight_grad(dz: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dW[o, c, k] = sum_{beam, n} dz[beam, n, o] x[beam, n + k - 4, c]."""
    nb, nr, _ = x.shape
    xp = np.zeros((nb, nr + 2 * HALF, x.shape[2]))
    xp[:, HALF:HALF + nr] = x
    dW = np.zeros((dz.shape[2], x.shape[2], KERNEL))
    for k in range(KERNEL):
        dW[:, :, k] = np.einsum("bno,bnc->oc", dz, xp[:, k:k + nr])
    return dW


def forward(net: dict, x0: np.ndarray, bf16_storage: bool = False):
    """Activations [a0 = x0, a1, ..., a5] and the output yhat [beams, n_range]."""
    acts = [np.asarray(x0, np.float64)]
    n_layers = len(net["W"])
    for l in range(n_layers):
        z = conv(acts[-1], net["W"][l], net["b"][l])
        if l < n_layers - 1:
            a = np.maximum(z, 0.0)
            acts.append(bf16(a) if bf16_storage else a)
        else:
            return acts, z[..., 0]


def loss(yhat: np.ndarray, y: np.ndarray) -> float:
    """Mean squared error over every (beam, bin)."""
    return float(np.mean((yhat - y) ** 2))


def backward(net: dict, acts: list, yhat: np.ndarray, y: np.ndarray, bf16_storage: bool = False):
    """Gradients of the mean squared error: lists dW, db (per layer)."""
    n_layers = len(net["W"])
    dW = [None] * n_layers
    db = [None] * n_layers
    dz = (2.0 * (yhat - y) / yhat.size)[..., None]
    for l in range(n_layers - 1, -1, -1):
        dW[l] = conv_weight_grad(dz, acts[l])
        db[l] = dz.sum(axis=(0, 1))
        if l == 0:
            break
        da = conv_input_grad(dz, net["W"][l])
        dz = da * (acts[l] > 0)
        if bf16_storage:
            dz = bf16(dz)
    return dW, db


def adam(theta, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) at step count t >= 1: returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ evaluation
def beam_metrics(E: np.ndarray, E_ref: np.ndarray, n_blank: int, rel_thr: float):
    """Per-ping evaluation of an envelope volume E [beams, n_range] against the plain
    method's E_ref. The ping maximum vmax is E_ref's largest value at or beyond bin
    n_blank. Returns a dict: normalised L2 error; the per-beam peak-bin error
    |argmax E - argmax E_ref| (bins at or beyond n_blank, first index on ties, negative
    values of E counted as zero) over the lit beams, whose E_ref peak is positive and
    reaches rel_thr vmax; and the speckle statistic of both volumes, the scintillation
    index var(I) / mean(I)^2 of the intensity I = E^2 over the (beam, bin) cells where
    E_ref is positive and reaches rel_thr vmax."""
    E = np.asarray(E, np.float64)
    E_ref = np.asarray(E_ref, np.float64)
    nl2 = float(np.linalg.norm(E - E_ref) / np.linalg.norm(E_ref))
    sub, sub_ref = np.maximum(E[:, n_blank:], 0.0), E_ref[:, n_blank:]
    vmax = sub_ref.max()
    bmax = sub_ref.max(axis=1)
    lit = (bmax >= rel_thr * vmax) & (bmax > 0)
    dpk = np.abs(np.argmax(sub, axis=1) - np.argmax(sub_ref, axis=1))[lit]
    cells = (E_ref >= rel_thr * vmax) & (E_ref > 0)

    def si(A):
        I = A[cells] ** 2
        return float(I.var() / I.mean() ** 2)

    return {"nl2": nl2, "peak_bins": dpk, "si": si(E), "si_ref": si(E_ref)}
