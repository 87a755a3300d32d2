"""Host-side arithmetic of bench.py (no GPU): the algorithmic bytes and propagator flops per site
of a coupled step that the step-level roofline fractions divide by."""
import bench


def test_step_bytes_per_site():
    # 128^3 workload: N = 64, 4 inversion iterations of 2 density evaluations, 8 Jacobi sweeps, LB
    assert bench.step_bytes_per_site(64, 4, 8, 1) == 8 * (8 * 64 + 64) + 24 + 44 + 40 * 8 + 180
    assert bench.step_bytes_per_site(64, 4, 8, 1, es=8) == 2 * bench.step_bytes_per_site(64, 4, 8, 1)
    assert bench.step_bytes_per_site(64, 4, 8, 0) == bench.step_bytes_per_site(64, 4, 8, 1) - 180
    assert bench.step_bytes_per_site(16, 6, 8, 1, evals_per_iter=1) == 6 * (8 * 16 + 64) + 24 + 44 + 320 + 180


def test_step_prop_flops_per_site():
    assert bench.step_prop_flops_per_site(64, 4) == 2 * 4 * 28 * 64
    assert bench.step_prop_flops_per_site(10, 1, evals_per_iter=1) == 280
