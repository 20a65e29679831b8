"""FP64 CPU oracle of the learned initial guess (message-passing network on coarse edges).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

The network predicts the PCG initial guess of the potential solve from the
right-hand side and the two previous solutions (the learned-guess addition
on top of the method of Sect. 2.2).  Per coarse node i the inputs are

    f_i = [r_i / s_r, (phi1 - phi2)_i / s_d, b_i / s_b, x_i / L, y_i / L]

with r = b - K phi(t-1) the residual of the previous solution for the new
right-hand side (K dphi = r drives the increment), s_r, s_d, s_b the rms
values over the nodes (floored), L = 15 the outer radius.  Each input is
scaled by its own size because BF16 activations (8-bit mantissa) cannot
resolve phi(t-1) against phi(t-2) when both are scaled by rms(phi).  For every directed mesh edge (i <- j) the edge feature is
e_ij = (dx, dy, |d|) / ell, d = x_j - x_i, ell the mean edge length.

    h0   = relu(We f + be)                                   (encoder, FP32)
    for l = 1..3:
      m_ij = relu(Wm_l [h_i ; h_j ; e_ij] + bm_l)             (per directed edge)
      a_i  = sum_{j in N(i)} m_ij
      h_i  = h_i + relu(Wu_l [h_i ; a_i] + bu_l)
    out_i = Wd h_i + bd
    x0    = phi1 + s_d * out                                 (then projected to mean zero)

Training target: t_i = (phi(t)_i - phi(t-1)_i) / s_d, loss = mean (out - t)^2:
the network predicts the next increment in units of the last one (linear
extrapolation is out = (phi1 - phi2) / s_d, a zero decoder gives phi1).
Activations h, messages m, aggregates a and the dense weights Wm, Wu are
stored in BF16 (round to nearest even) where the GPU stores them; every sum
is exact FP64 here.  ``bf16=False`` gives the plain FP64 network used for
the finite-difference check.  Adam: lr 1e-3, betas (0.9, 0.999), eps 1e-8.
"""
from __future__ import annotations

import numpy as np

H = 64
N_LAYERS = 3
F_IN = 5
E_FEAT = 3
R_OUT = 15.0


def bf16(x):
    """Round float64/float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out.reshape(np.shape(x))


def param_shapes():
    shapes = {"We": (H, F_IN), "be": (H,)}
    for l in range(N_LAYERS):
        shapes[f"Wm{l}"] = (H, 2 * H + E_FEAT)
        shapes[f"bm{l}"] = (H,)
        shapes[f"Wu{l}"] = (H, 2 * H)
        shapes[f"bu{l}"] = (H,)
    shapes["Wd"] = (1, H)
    shapes["bd"] = (1,)
    return shapes


def init_params(seed: int = 0, zero_decoder: bool = True):
    """He-normal weights, zero biases; a zero decoder makes the initial guess phi(t-1)."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in param_shapes().items():
        if k.startswith("W"):
            fan_in = shp[1]
            p[k] = rng.standard_normal(shp) * np.sqrt(2.0 / fan_in)
        else:
            p[k] = np.zeros(shp)
    if zero_decoder:
        p["Wd"][:] = 0.0
    return p


class Graph:
    """Directed edges (i <- j) of a mesh in CSR order of the destination i, with edge features."""

    def __init__(self, K_csr, xy):
        indptr, indices = K_csr.indptr, K_csr.indices
        n = xy.shape[0]
        dst, src = [], []
        for i in range(n):
            for k in range(indptr[i], indptr[i + 1]):
                j = indices[k]
                if j != i:
                    dst.append(i)
                    src.append(j)
        self.n = n
        self.dst = np.array(dst, dtype=np.int64)
        self.src = np.array(src, dtype=np.int64)
        d = xy[self.src] - xy[self.dst]
        length = np.sqrt(np.sum(d * d, axis=1))
        self.ell = float(np.mean(length))
        self.efeat = np.stack([d[:, 0], d[:, 1], length], axis=1) / self.ell
        self.xy = xy


def rms(v):
    return float(np.sqrt(np.mean(np.asarray(v) ** 2)))


def floor_scale(s):
    return s if s > 1e-30 else 1.0


def features(g: Graph, K, b, phi1, phi2):
    """Input features and the output scale s_d = rms(phi1 - phi2)."""
    r = b - K @ phi1
    d = phi1 - phi2
    s_r = floor_scale(rms(r))
    s_d = floor_scale(rms(d))
    s_b = floor_scale(rms(b))
    f = np.stack([r / s_r, d / s_d, b / s_b, g.xy[:, 0] / R_OUT, g.xy[:, 1] / R_OUT], axis=1)
    return f, s_d


def forward(p, g: Graph, f, bf16_storage=True):
    """Forward pass; returns (out [n], cache for backward)."""
    rd = bf16 if bf16_storage else (lambda v: np.asarray(v, dtype=np.float64))
    e = rd(g.efeat)
    cache = {"f": f, "e": e}
    z0 = f @ p["We"].T + p["be"]
    h = rd(np.maximum(z0, 0.0))
    cache["z0"] = z0
    cache["h"] = [h]
    for l in range(N_LAYERS):
        Wm, Wu = rd(p[f"Wm{l}"]), rd(p[f"Wu{l}"])
        x_e = np.concatenate([h[g.dst], h[g.src], e], axis=1)
        z = x_e @ Wm.T + p[f"bm{l}"]
        m = rd(np.maximum(z, 0.0))
        a_exact = np.zeros((g.n, H))
        np.add.at(a_exact, g.dst, m)
        a = rd(a_exact)
        x_n = np.concatenate([h, a], axis=1)
        u = x_n @ Wu.T + p[f"bu{l}"]
        h_new = rd(h + np.maximum(u, 0.0))
        cache[f"L{l}"] = dict(x_e=x_e, z=z, a=a, x_n=x_n, u=u, Wm=Wm, Wu=Wu)
        h = h_new
        cache["h"].append(h)
    out = h @ p["Wd"][0] + p["bd"][0]
    return out, cache


def loss_and_grad(p, g: Graph, samples, bf16_storage=True):
    """Mean squared error over all nodes of all samples and its gradient w.r.t. every parameter.

    samples: list of (f [n,5], target [n]).  Straight-through for the BF16
    rounding: the backward pass differentiates the unrounded operations and
    uses the rounded tensors where the forward used them.
    """
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    total = 0.0
    count = sum(s[0].shape[0] for s in samples)
    for f, t in samples:
        out, c = forward(p, g, f, bf16_storage)
        diff = out - t
        total += float(np.sum(diff * diff))
        dout = 2.0 * diff / count
        h = c["h"][-1]
        grads["Wd"][0] += dout @ h
        grads["bd"][0] += np.sum(dout)
        dh = np.outer(dout, p["Wd"][0])
        for l in reversed(range(N_LAYERS)):
            L = c[f"L{l}"]
            du = dh * (L["u"] > 0)
            grads[f"Wu{l}"] += du.T @ L["x_n"]
            grads[f"bu{l}"] += du.sum(axis=0)
            dxn = du @ L["Wu"]
            dh_prev = dh + dxn[:, :H]
            da = dxn[:, H:]
            dm = da[g.dst]
            dz = dm * (L["z"] > 0)
            grads[f"Wm{l}"] += dz.T @ L["x_e"]
            grads[f"bm{l}"] += dz.sum(axis=0)
            dxe = dz @ L["Wm"]
            np.add.at(dh_prev, g.dst, dxe[:, :H])
            np.add.at(dh_prev, g.src, dxe[:, H:2 * H])
            dh = dh_prev
        dz0 = dh * (c["z0"] > 0)
        grads["We"] += dz0.T @ c["f"]
        grads["be"] += dz0.sum(axis=0)
    return total / count, grads


def magnitudes(p, g: Graph, samples, bf16_storage=True):
    """Size of the terms behind every output and gradient element, for elementwise bounds.

    The same forward and backward passes as ``forward`` and
    ``loss_and_grad`` with every weight, input and intermediate replaced by
    its absolute value, so each returned element is the sum of the absolute
    values of all the products that make up the corresponding element of the
    network (relu(a) - relu(b) is bounded by a - b, so activations carry the
    magnitude of their argument).  A relative perturbation eps of every
    stored value changes an output or gradient element by at most about
    eps times its magnitude.  The backward keeps the relu masks of the
    rounded forward.  Returns (list of [n] output magnitudes, dict of
    gradient magnitudes).
    """
    mags = {k: np.zeros_like(v) for k, v in p.items()}
    outs = []
    count = sum(s[0].shape[0] for s in samples)
    A = {k: np.abs(v) for k, v in p.items()}
    rd = bf16 if bf16_storage else (lambda v: np.asarray(v, dtype=np.float64))
    for f, t in samples:
        _, c = forward(p, g, f, bf16_storage)
        e = np.abs(c["e"])
        Mh = np.abs(f) @ A["We"].T + A["be"]
        Mhs = [Mh]
        ML = []
        for l in range(N_LAYERS):
            Wm, Wu = np.abs(rd(p[f"Wm{l}"])), np.abs(rd(p[f"Wu{l}"]))
            Mxe = np.concatenate([Mh[g.dst], Mh[g.src], e], axis=1)
            Mm = Mxe @ Wm.T + A[f"bm{l}"]
            Ma = np.zeros((g.n, H))
            np.add.at(Ma, g.dst, Mm)
            Mxn = np.concatenate([Mh, Ma], axis=1)
            Mu = Mxn @ Wu.T + A[f"bu{l}"]
            ML.append(dict(Mxe=Mxe, Mxn=Mxn, Wm=Wm, Wu=Wu))
            Mh = Mh + Mu
            Mhs.append(Mh)
        Mout = Mh @ A["Wd"][0] + A["bd"][0]
        outs.append(Mout)
        Mdout = 2.0 * (Mout + np.abs(t)) / count
        mags["Wd"][0] += Mdout @ Mh
        mags["bd"][0] += np.sum(Mdout)
        Mdh = np.outer(Mdout, A["Wd"][0])
        for l in reversed(range(N_LAYERS)):
            L, M = c[f"L{l}"], ML[l]
            Mdu = Mdh * (L["u"] > 0)
            mags[f"Wu{l}"] += Mdu.T @ M["Mxn"]
            mags[f"bu{l}"] += Mdu.sum(axis=0)
            Mdxn = Mdu @ M["Wu"]
            Mdh_prev = Mdh + Mdxn[:, :H]
            Mdz = Mdxn[:, H:][g.dst] * (L["z"] > 0)
            mags[f"Wm{l}"] += Mdz.T @ M["Mxe"]
            mags[f"bm{l}"] += Mdz.sum(axis=0)
            Mdxe = Mdz @ M["Wm"]
            np.add.at(Mdh_prev, g.dst, Mdxe[:, :H])
            np.add.at(Mdh_prev, g.src, Mdxe[:, H:2 * H])
            Mdh = Mdh_prev
        Mdz0 = Mdh * (c["z0"] > 0)
        mags["We"] += Mdz0.T @ np.abs(c["f"])
        mags["be"] += Mdz0.sum(axis=0)
    return outs, mags


class Adam:
    def __init__(self, p, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in p.items()}
        self.v = {k: np.zeros_like(v) for k, v in p.items()}
        self.t = 0

    def step(self, p, grads):
        self.t += 1
        for k in p:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * grads[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * grads[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            p[k] = p[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def guess(p, g: Graph, K, b, phi1, phi2, bf16_storage=True):
    """Initial guess phi1 + s_d * out, projected to mean zero."""
    f, s_d = features(g, K, b, phi1, phi2)
    out, _ = forward(p, g, f, bf16_storage)
    x0 = phi1 + s_d * out
    return x0 - x0.mean()
