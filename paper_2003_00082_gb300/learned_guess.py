"""Training and evaluation of the learned PCG initial guess (the message-passing network).

Training data are potential solves produced by the method itself: for every
(Stuart number, seed) pair a sequence of time steps of the advected vortex
train with noise is solved with FP64 PCG (previous-step initial guess,
tolerance 1e-8), and each step t >= 2 gives one sample
(b(t), phi(t-1), phi(t-2)) -> phi(t).  The electric potential of Eq. 12 does
not depend on the conductivity, so the Stuart number only changes the
force; samples of different N for the same seed repeat the same potentials.

Evaluation runs held-out seeds and compares, at the same tolerance, the PCG
iterations and solves per second of two initial guesses: phi(t-1) (the
method without the network) and the network's prediction.
"""
from __future__ import annotations

import time

import numpy as np

from . import cgp, inputs

H = 64
N_LAYERS = 3
F_IN = 5
E_FEAT = 3


def param_shapes():
    """Parameter order and shapes of the network (the C ABI's packed layout)."""
    shapes = {"We": (H, F_IN), "be": (H,)}
    for l in range(N_LAYERS):
        shapes[f"Wm{l}"] = (H, 2 * H + E_FEAT)
        shapes[f"bm{l}"] = (H,)
        shapes[f"Wu{l}"] = (H, 2 * H)
        shapes[f"bu{l}"] = (H,)
    shapes["Wd"] = (1, H)
    shapes["bd"] = (1,)
    return shapes


def initial_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases and a zero decoder (the untrained guess is phi(t-1))."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, shp in param_shapes().items():
        if k.startswith("W") and k != "Wd":
            parts.append((rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])).reshape(-1))
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    return np.concatenate(parts).astype(np.float32)


def solve_sequence(torch, mesh, xy_f, seed, steps, B=(0.0, 0.0, 1.0), noise_std=1e-3, tol=1e-8, dev="cuda"):
    """Potential solves of one trajectory on the GPU: returns (b [steps, n], phi [steps, n], iterations)."""
    n = mesh.n_c
    f64 = dict(dtype=torch.float64, device=dev)
    b_all = torch.empty((steps, n), **f64)
    phi_all = torch.empty((steps, n), **f64)
    x = torch.zeros(n, **f64)
    its = []
    for t in range(steps):
        u, v = inputs.velocity(xy_f, t, seed, vortices=True, noise_std=noise_std)
        cgp.cgp_restrict(mesh.handle, cgp.CGP_RHS_POTENTIAL, B, 20.0, torch.as_tensor(u, device=dev),
                         torch.as_tensor(v, device=dev), b_all[t])
        info = cgp.cgp_poisson_solve(mesh.handle, b_all[t], x, tol=tol, use_x0=t > 0)
        if info["status"] != cgp.CGP_OK:
            raise RuntimeError(f"solve failed: {info}")
        its.append(info["iterations"])
        phi_all[t].copy_(x)
    return b_all, phi_all, its


def make_samples(torch, seqs):
    """Stack (b(t), phi(t-1), phi(t-2), phi(t)) for t >= 2 over all sequences."""
    b = torch.cat([s[0][2:] for s in seqs])
    p1 = torch.cat([s[1][1:-1] for s in seqs])
    p2 = torch.cat([s[1][:-2] for s in seqs])
    pt = torch.cat([s[1][2:] for s in seqs])
    return b, p1, p2, pt


def train(torch, net, samples, iterations=1500, batch=16, lr=1e-3, seed=0, dev="cuda"):
    """Adam on random minibatches; returns the loss of every 50th step."""
    b, p1, p2, pt = samples
    count = b.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    loss_dev = torch.zeros(1, dtype=torch.float32, device=dev)
    for it in range(iterations):
        idx = torch.as_tensor(rng.choice(count, size=batch, replace=False), device=dev)
        net.train_step(batch, b[idx].contiguous(), p1[idx].contiguous(), p2[idx].contiguous(),
                       pt[idx].contiguous(), lr=lr, loss_dev=loss_dev)
        if it % 50 == 0 or it == iterations - 1:
            losses.append(float(loss_dev.item()))
    return losses


def evaluate(torch, mesh, net, xy_f, seeds, steps, B=(0.0, 0.0, 1.0), noise_std=1e-3, tol=1e-8, dev="cuda"):
    """Held-out trajectories solved with three initial guesses: phi(t-1) (the method
    without the network), the linear extrapolation 2 phi(t-1) - phi(t-2), and the
    network's guess.

    All runs solve the same right-hand sides to the same tolerance.  Solves are
    launched without host synchronisation and timed on the device with CUDA
    events (the learned run's time includes the network's inference).  Returns
    mean iteration counts, solves per second of the previous-step and learned
    runs, and the largest relative difference between their solutions.
    """
    n = mesh.n_c
    f64 = dict(dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    base_its, learn_its, extrap_its = [], [], []
    ms_base = ms_learn = 0.0
    worst = 0.0
    for seed in seeds:
        b_all = torch.empty((steps, n), **f64)
        for t in range(steps):
            u, v = inputs.velocity(xy_f, t, seed, vortices=True, noise_std=noise_std)
            cgp.cgp_restrict(mesh.handle, cgp.CGP_RHS_POTENTIAL, B, 20.0, torch.as_tensor(u, device=dev),
                             torch.as_tensor(v, device=dev), b_all[t])
        infos = torch.zeros(3 * steps * cgp.INFO_BYTES, dtype=torch.uint8, device=dev)
        slot = lambda k: infos.data_ptr() + k * cgp.INFO_BYTES  # noqa: E731
        events = []
        # baseline: previous-step guess
        phi_base = torch.zeros((steps, n), **f64)
        x = torch.zeros(n, **f64)
        for t in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cgp.cgp_poisson_solve_async(mesh.handle, b_all[t], x, tol=tol, use_x0=t > 0, info_dev=slot(t))
            e1.record(stream)
            phi_base[t].copy_(x)
            if t >= 2:
                events.append(("base", e0, e1))
        # linear extrapolation 2 phi(t-1) - phi(t-2), for context
        xe = torch.empty(n, **f64)
        for t in range(2, steps):
            xe.copy_(2.0 * phi_base[t - 1] - phi_base[t - 2])
            cgp.cgp_poisson_solve_async(mesh.handle, b_all[t], xe, tol=tol, use_x0=True, info_dev=slot(steps + t))
        # learned guess from step 2 on (the network needs two previous solutions)
        phi = torch.zeros((steps, n), **f64)
        phi[0].copy_(phi_base[0])
        phi[1].copy_(phi_base[1])
        for t in range(2, steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.predict(b_all[t], phi[t - 1], phi[t - 2], phi[t])
            cgp.cgp_poisson_solve_async(mesh.handle, b_all[t], phi[t], tol=tol, use_x0=True,
                                        info_dev=slot(2 * steps + t))
            e1.record(stream)
            events.append(("learn", e0, e1))
        torch.cuda.synchronize()
        for kind, e0, e1 in events:
            if kind == "base":
                ms_base += e0.elapsed_time(e1)
            else:
                ms_learn += e0.elapsed_time(e1)
        recs = cgp.decode_infos(bytes(infos.cpu().numpy()), 3 * steps)
        for t in range(2, steps):
            for r in (recs[t], recs[steps + t], recs[2 * steps + t]):
                if r["status"] != cgp.CGP_OK:
                    raise RuntimeError(f"solve failed: {r}")
            base_its.append(recs[t]["iterations"])
            extrap_its.append(recs[steps + t]["iterations"])
            learn_its.append(recs[2 * steps + t]["iterations"])
            d = float(torch.linalg.norm(phi[t] - phi_base[t]) / torch.linalg.norm(phi_base[t]))
            worst = max(worst, d)
    return dict(baseline_iterations_mean=float(np.mean(base_its)), learned_iterations_mean=float(np.mean(learn_its)),
                extrapolation_iterations_mean=float(np.mean(extrap_its)),
                baseline_solves_per_s=len(base_its) / (ms_base * 1e-3),
                learned_solves_per_s=len(learn_its) / (ms_learn * 1e-3),
                max_rel_diff_between_runs=worst, solves=len(base_its))


def run_protocol(torch, mesh, xy_f, train_seeds=(0, 1, 2, 3, 4), train_stuart=(0.5, 1.0, 2.0, 5.0), steps=200,
                 test_seeds=(100, 101, 102, 103, 104), test_steps=200, iterations=(2000, 1000), lrs=(1e-3, 3e-4),
                 batch=32, seed=0, noise_std=1e-3):
    """Generate training solves, train the network, evaluate on held-out seeds."""
    t0 = time.perf_counter()
    seqs = {}
    for stuart in train_stuart:           # the potential does not depend on N: solved per N as the protocol asks
        for s in train_seeds:
            seqs[(stuart, s)] = solve_sequence(torch, mesh, xy_f, s, steps, noise_std=noise_std)
    gen_s = time.perf_counter() - t0
    distinct = [seqs[(train_stuart[0], s)] for s in train_seeds]
    samples = make_samples(torch, distinct)
    net = cgp.GNN(mesh, batch, initial_params(seed))
    t0 = time.perf_counter()
    losses = []
    for iters, lr in zip(iterations, lrs):
        losses += train(torch, net, samples, iterations=iters, batch=batch, lr=lr, seed=seed)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    ev = evaluate(torch, mesh, net, xy_f, test_seeds, test_steps, noise_std=noise_std)
    ev.update(training_solves=len(seqs) * steps, distinct_samples=int(samples[0].shape[0]),
              generation_seconds=gen_s, training_seconds=train_s, loss_first=losses[0], loss_last=losses[-1],
              train_iterations=int(sum(iterations)))
    return net, ev
