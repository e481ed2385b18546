"""The warp-per-point solve (solve variants 22-24: one warp per Gauss point,
lane l condensing the subtree under level-6 node l in registers) against the
FP64 oracle, at the mixed path's tolerances of test_gpu_parity: every depth it
serves, plastic increments with several Newton iterations, line-search
backtracking, the benchmark's 65,536-point batch (sampled), the warm start
with its fallback, and bit-reproducibility."""
import numpy as np
import pytest

from paper_2109_14403_gb300 import synthetic as syn
from test_gpu_parity import TOL_WARM, _dev, compare, run_path  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WARP = [22, 23, 24]


@pytest.mark.parametrize("K", [6, 7, 8])
@pytest.mark.parametrize("variant", WARP)
def test_warp_kernel_depths(K, variant):
    rng = np.random.default_rng(300 + K)
    n = 37
    deps = rng.normal(0, 3e-3, size=(3, n, 6))
    theta = 293.0 + np.cumsum(rng.uniform(0, 5, size=(3, n)), axis=0)
    run_path(K, "mixed", deps, theta, dt=0.7, variant=variant)


@pytest.mark.parametrize("variant", WARP)
def test_warp_kernel_k8_backtracking_walk(variant):
    """Scaled K=8 random walk: several Newton iterations and, at some points,
    rejected full steps (line-search backtracking)."""
    deps, theta = syn.random_walk_k8(n_points=200, n_incr=2)
    run_path(8, "mixed", deps * 20.0, theta, variant=variant)


@pytest.mark.parametrize("variant", WARP)
def test_warp_kernel_k8_plastic_walk(variant):
    deps, theta = syn.random_walk_k8(n_points=200, n_incr=4)
    run_path(8, "mixed", deps * 8.0, theta, variant=variant)


def test_warp_kernel_k8_full_batch_sampled():
    """The benchmark's batch size (65,536 points, every CTA slot busy, ragged
    last wave); the oracle checks 96 sampled points."""
    deps, theta = syn.random_walk_k8(n_points=65536, n_incr=2)
    run_path(8, "mixed", deps, theta, n_check=96, variant=23)


@pytest.mark.parametrize("variant", WARP)
def test_warp_kernel_warm_start_and_fallback(variant):
    """dmn_eval_warm on the warp form (K = 6): non-finite starts fall back to
    a^n in the same launch, zero starts equal the plain path, perturbed
    oracle increments converge within the stopping-criterion bound."""
    import test_gpu_parity as tp
    tp.test_warm_start_parity_and_fallback("mixed", variant)


def test_warp_kernel_deterministic_bits():
    from paper_2109_14403_gb300 import DMN
    dev = _dev()
    w, nrm, ph = syn.tree(8)
    d = DMN(8, w, nrm, ph, syn.materials(), precision="mixed", solve_variant=23)
    deps, theta = syn.random_walk_k8(n_points=3000, n_incr=1)
    dd = torch.tensor(deps[0] * 8, device=dev)
    th = torch.tensor(theta[0], device=dev)
    s = d.init_state(torch.full((3000,), 293.0, dtype=torch.float64, device=dev))
    r1 = d.eval(dd, th, 1.0, s)
    r2 = d.eval(dd, th, 1.0, s)
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    d.close()


def test_warp_variant_rejected_where_unsupported():
    from paper_2109_14403_gb300 import DMN
    _dev()
    w, nrm, ph = syn.tree(5)
    with pytest.raises(RuntimeError, match="one warp per point"):
        DMN(5, w, nrm, ph, syn.materials(), precision="mixed", solve_variant=23)
    w, nrm, ph = syn.tree(8)
    with pytest.raises(RuntimeError, match="one warp per point"):
        DMN(8, w, nrm, ph, syn.materials(), precision="fp64", solve_variant=23)
