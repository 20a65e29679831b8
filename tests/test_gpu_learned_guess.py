"""What the trained network gains over the method without it (previous-step initial guess).

Trains the network with the project's GPU kernels on potential solves the
method produces on the 64x32 mesh (vortex train with noise, seeds 0-4), then
solves held-out trajectories (seeds 100-101) to the same 1e-8 tolerance with
both initial guesses.  The learned guess must need fewer PCG iterations and
give the same solution.
"""
import pytest

from paper_2003_00082_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_trained_network_reduces_pcg_iterations():
    from paper_2003_00082_gb300 import build, cgp, learned_guess as LG
    build.build()
    cgp.load()
    xy, tri = inputs.ogrid(64, 32)
    m = cgp.Mesh(xy, tri)
    xy_f, _, _ = m.fine_geometry()
    net, ev = LG.run_protocol(torch, m, xy_f, train_stuart=(1.0,), steps=200, test_seeds=(100, 101), test_steps=100,
                              iterations=(1500, 500))
    print(ev)
    assert ev["loss_last"] < 0.5 * ev["loss_first"]
    assert ev["learned_iterations_mean"] < ev["baseline_iterations_mean"]
    assert ev["max_rel_diff_between_runs"] <= 1e-6
    net.close()
    m.close()


def test_trained_network_beats_the_previous_step_guess_on_a_smooth_sequence():
    """Without the per-step noise (the benchmark's own velocity sequence) most of the step-to-step
    change is predictable: the trained guess must save at least 15 % of the PCG iterations and
    beat linear extrapolation, with the same solution."""
    from paper_2003_00082_gb300 import build, cgp, learned_guess as LG
    build.build()
    cgp.load()
    xy, tri = inputs.ogrid(128, 64)
    m = cgp.Mesh(xy, tri)
    xy_f, _, _ = m.fine_geometry()
    net, ev = LG.run_protocol(torch, m, xy_f, train_seeds=(0, 1, 2), train_stuart=(1.0,), steps=100,
                              test_seeds=(100,), test_steps=40, iterations=(600, 300), batch=8, noise_std=0.0)
    print(ev)
    assert ev["learned_iterations_mean"] <= 0.85 * ev["baseline_iterations_mean"]
    assert ev["learned_iterations_mean"] < ev["extrapolation_iterations_mean"]
    assert ev["max_rel_diff_between_runs"] <= 1e-6
    net.close()
    m.close()
