"""Batched persistent solves of uneven systems: each instance against the CPU oracle."""
import numpy as np
import pytest

from oracle import cgp_oracle as O
from paper_2003_00082_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def cgp():
    from paper_2003_00082_gb300 import build, cgp as c
    build.build()
    c.load()
    return c


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def rel(a, r):
    return float(np.linalg.norm(np.asarray(a) - r) / np.linalg.norm(r))


# uneven sizes up to the two largest of the 64-instance workload (256x128 and 512x256: in the
# wave schedule a 512x256 system gets the whole GPU, in the packed one a share of a single launch)
SIZES = [(8, 4), (16, 8), (33, 17), (64, 32), (128, 64), (7, 3), (96, 48), (256, 128), (512, 256)]


@pytest.fixture(scope="module")
def systems(cgp):
    out = []
    for k, (nt, nr) in enumerate(SIZES):
        xy, tri = inputs.ogrid(nt, nr)
        m = cgp.Mesh(xy, tri)
        om = O.OracleMesh(xy, tri)
        u, v = inputs.velocity(om.xy_f, k, 7, vortices=True, noise_std=1e-3)
        ang = 0.7 * k
        B = (np.cos(ang), np.sin(ang), 1.0)
        Fx, Fy = O.source_field(O.POTENTIAL, om.restrict(u), om.restrict(v), B)
        b = O.rhs(om.Gx, om.Gy, Fx, Fy)
        exact = O.pcg(om.K, om.d, b, tol=1e-13, max_it=8000)["x"]   # far below the tests' 1e-7
        out.append(dict(mesh=m, om=om, b=b, exact=exact))
    yield out
    for s in out:
        s["mesh"].close()


@pytest.mark.parametrize("packed", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_batched_instances_match_the_oracle(cgp, systems, precision, packed):
    bs = [T(s["b"]) for s in systems]
    xs = [torch.zeros_like(b) for b in bs]
    batch = cgp.Batch([s["mesh"] for s in systems], bs, xs, tol=1e-10, precision=precision)
    if packed:   # one launch holding every system
        batch.set_tuning(512, 1, 0, 4)
    q = batch.query()
    if packed:
        assert q["grid"] == sum(q["blocks"])
    else:        # waves: each system gets what it would get alone (about 256 rows a block, one SM's worth at most)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert q["grid"] <= sum(q["blocks"])
        assert q["blocks"] == [min(sms, max(1, (s["mesh"].n_c + 255) // 256)) for s in systems]
    assert min(q["blocks"]) >= 1
    batch.solve()
    infos, secs = batch.info()
    for s, x, info, t in zip(systems, xs, infos, secs):
        assert info["status"] == cgp.CGP_OK, info
        assert info["rel_res_true"] <= 1.1e-10
        assert rel(x.cpu().numpy(), s["exact"]) <= 1e-7
        assert t > 0.0
    sizes = [s["mesh"].n_c for s in systems]
    small, large = int(np.argmin(sizes)), int(np.argmax(sizes))
    if packed:   # the largest system should not finish before the smallest
        assert max(secs) >= min(secs)
    else:        # the wave of the smallest systems runs first, the 512x256 system's own wave last
        assert secs[small] < secs[large]
    batch.close()


@pytest.mark.parametrize("block,lanes,per_sm,flags", [(256, 1, 1, 0), (512, 2, 2, 1), (128, 4, 0, 0), (64, 8, 1, 1),
                                                     (256, 1, 1, 4), (512, 2, 2, 5), (256, 1, 2, 2), (128, 1, 0, 6),
                                                     (256, 1, 1, 8), (512, 1, 1, 12), (128, 2, 0, 9),
                                                     (256, 1, 1, 16), (512, 2, 1, 20), (256, 4, 1, 20),
                                                     (512, 1, 1, 32), (512, 1, 1, 64), (256, 2, 1, 96),
                                                     (512, 1, 1, 72), (512, 2, 1, 96)])
def test_batched_launch_shapes(cgp, systems, block, lanes, per_sm, flags):
    bs = [T(s["b"]) for s in systems]
    xs = [torch.zeros_like(b) for b in bs]
    batch = cgp.Batch([s["mesh"] for s in systems], bs, xs, tol=1e-10)
    batch.set_tuning(block, lanes, per_sm, flags)
    q = batch.query()
    assert q["block"] == block and q["lanes"] == lanes
    if flags & 1:
        assert q["resident"] == 0
    if flags & 96 and not flags & 4:   # waves of 256 << k rows a block, no fewer blocks than that asks
        rows = 256 << ((flags >> 5) & 3)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for s, nb in zip(systems, q["blocks"]):
            n = s["mesh"].n_c
            assert min(sms, -(-n // rows)) <= nb <= min(sms, max(1, -(-n // 256)))
    batch.solve()
    infos, _ = batch.info()
    for s, x, info in zip(systems, xs, infos):
        assert info["status"] == cgp.CGP_OK
        assert rel(x.cpu().numpy(), s["exact"]) <= 1e-7
    batch.close()


@pytest.mark.parametrize("block,lanes,per_sm,flags", [(512, 1, 1, 8), (512, 1, 1, 104), (256, 2, 1, 8), (512, 1, 0, 12)])
def test_batched_mixed_tagged_shapes(cgp, systems, block, lanes, per_sm, flags):
    """Mixed precision with tagged FP32 inner reductions (flag bit 3), alone, with 2048 rows a block and in
    one packed launch: every instance still reaches the oracle's answer."""
    bs = [T(s["b"]) for s in systems]
    xs = [torch.zeros_like(b) for b in bs]
    batch = cgp.Batch([s["mesh"] for s in systems], bs, xs, tol=1e-10, precision=cgp.CGP_MIXED)
    batch.set_tuning(block, lanes, per_sm, flags)
    batch.solve()
    infos, _ = batch.info()
    for s, x, info in zip(systems, xs, infos):
        assert info["status"] == cgp.CGP_OK, info
        assert info["rel_res_true"] <= 1.1e-10
        assert rel(x.cpu().numpy(), s["exact"]) <= 1e-7
    batch.close()


def test_batched_solve_replays_in_a_cuda_graph(cgp, systems):
    bs = [T(s["b"]) for s in systems]
    xs = [torch.zeros_like(b) for b in bs]
    batch = cgp.Batch([s["mesh"] for s in systems], bs, xs, tol=1e-10, precision=cgp.CGP_MIXED)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        batch.solve()
    for rep in range(2):
        for x in xs:
            x.zero_()
        g.replay()
        torch.cuda.synchronize()
        infos, _ = batch.info()
        for s, x, info in zip(systems, xs, infos):
            assert info["status"] == cgp.CGP_OK
            assert rel(x.cpu().numpy(), s["exact"]) <= 1e-7
    batch.close()


def test_batch_autotune_keeps_results_correct(cgp, systems):
    bs = [T(s["b"]) for s in systems[:4]]
    xs = [torch.zeros_like(b) for b in bs]
    batch = cgp.Batch([s["mesh"] for s in systems[:4]], bs, xs, tol=1e-10)
    best = batch.autotune()
    assert best > 0.0
    for x in xs:
        x.zero_()
    batch.solve()
    infos, _ = batch.info()
    for s, x, info in zip(systems[:4], xs, infos):
        assert info["status"] == cgp.CGP_OK
        assert rel(x.cpu().numpy(), s["exact"]) <= 1e-7
    batch.close()


def test_one_shot_batched_call_and_argument_checks(cgp, systems):
    bs = [T(s["b"]) for s in systems[:3]]
    xs = [torch.zeros_like(b) for b in bs]
    infos = cgp.cgp_poisson_solve_batched([s["mesh"] for s in systems[:3]], bs, xs, tol=1e-10)
    assert all(i["status"] == cgp.CGP_OK for i in infos)
    with pytest.raises(cgp.CgpError) as e:
        cgp.Batch([systems[0]["mesh"], systems[0]["mesh"]], bs[:1] * 2, xs[:1] * 2)
    assert e.value.status == cgp.CGP_ERR_INVALID_ARG
