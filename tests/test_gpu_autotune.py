"""GPU checks of the sampled direct sum and of the autotuner, through the C ABI.

The sampled direct sum is the plain definition evaluated on the GPU in FP64;
it must agree with the CPU oracle to 1e-12 relative (rounding of the ~N-term
sums in a different order).  The autotuner's choice must meet the digit
setting against the oracle (rel-L2 <= 1e-3 or <= 1e-6), and its own sampled
estimate must be within its goal.
"""
import numpy as np
import pytest

import oracle
import paper_1711_02976_gb300 as rp
import synth
from gpu_util import cuda_tensor

pytestmark = pytest.mark.gpu


def test_direct_sampled_matches_oracle_one_system():
    sysm = synth.config1()
    tg = np.array([0, 1, 7, 100, 2048, 4095], dtype=np.int64)
    u = rp.rpy_direct_sampled(cuda_tensor(sysm.pos), [0, sysm.n], [sysm.a], cuda_tensor(sysm.f), sysm.s, tg)
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_direct_sampled_forest_systems_do_not_interact():
    a_sys = synth.uniform_cube(3000, seed=21, a=0.01)
    b_sys = synth.sphere_plus_cube(5000, seed=22, a=0.003)
    pos = np.concatenate([a_sys.pos, b_sys.pos])
    f = np.concatenate([a_sys.f, b_sys.f])
    off = [0, a_sys.n, a_sys.n + b_sys.n]
    s = [a_sys.s, 2.0 * b_sys.s]
    tg = np.array([5, 2999, 3000, 4444, 7999], dtype=np.int64)
    u = rp.rpy_direct_sampled(cuda_tensor(pos), off, [a_sys.a, b_sys.a], cuda_tensor(f), s, tg)
    ra = oracle.rpy_direct(a_sys.pos, a_sys.f, a_sys.a, a_sys.s, targets=tg[:2])
    rb = oracle.rpy_direct(b_sys.pos, b_sys.f, b_sys.a, 2.0 * b_sys.s, targets=tg[2:] - a_sys.n)
    ref = np.concatenate([ra, rb])
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_direct_sampled_coincident_beads():
    pos = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5005], [0.9, 0.1, 0.2]])
    f = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.0], [1.0, 1.0, 1.0]])
    a, s = 0.001, 1.0
    tg = np.arange(4, dtype=np.int64)
    u = rp.rpy_direct_sampled(cuda_tensor(pos), [0, 4], [a], cuda_tensor(f), s, tg)
    ref = oracle.rpy_direct(pos, f, a, s)
    assert np.max(np.abs(u - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("digits,precision", [(3, rp.RPY_FP64), (6, rp.RPY_FP64), (3, rp.RPY_FP32)])
def test_autotune_choice_meets_the_setting(digits, precision):
    sysm = synth.sphere_plus_cube(60000, seed=31, a=4e-4)
    P, F = cuda_tensor(sysm.pos), cuda_tensor(sysm.f)
    res = rp.rpy_autotune(P, [0, sysm.n], [sysm.a], F, sysm.s, digits, precision, n_samples=200, timed_reps=2)
    best = res["best"]
    bound = 1e-3 if digits == 3 else 1e-6
    assert best["digits"] == digits and best["precision"] == precision
    assert best["order_p"] > 0 and best["leaf_cap"] >= 8
    assert res["est_rel_l2"] <= res["goal"] <= bound
    assert res["matvec_ms"] > 0 and len(res["trials"]) >= 6
    assert all(t["status"] == 0 for t in res["trials"])
    # the chosen parameters against the oracle on other targets
    t = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], digits, leaf_cap=best["leaf_cap"], precision=precision,
                            order_p=best["order_p"], direct_w=best["direct_w"], direct_x=best["direct_x"])
    import torch
    U = torch.empty_like(F)
    rp.rpy_forest_matvec(t, F, [sysm.s], U)
    rp.rpy_tree_sync(t)
    tg = synth.sample_targets(sysm.n, k=300, seed=77)
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg)
    err = oracle.rel_l2(U.cpu().numpy()[tg], ref)
    assert err <= bound, (err, best)
    t.close()


def test_evaluate_sources_at_targets():
    """rpy_evaluate against the oracle on the union of sources and (force-free) targets,
    with targets on top of sources and within 2a of them."""
    rng = np.random.default_rng(41)
    src = synth.uniform_cube(6000, seed=42, a=0.003)
    tgt = rng.random((1500, 3))
    tgt[:5] = src.pos[:5]                              # on a source
    tgt[5:10] = src.pos[5:10] + 0.001                  # within 2a of a source
    import torch
    U = torch.empty((len(tgt), 3), dtype=torch.float64, device="cuda")
    rp.rpy_evaluate(cuda_tensor(src.pos), cuda_tensor(src.f), cuda_tensor(tgt), src.a, src.s, 6, U)
    pos = np.concatenate([src.pos, tgt])
    f = np.concatenate([src.f, np.zeros_like(tgt)])
    ref = oracle.rpy_direct(pos, f, src.a, src.s, targets=np.arange(src.n, src.n + len(tgt)))
    u = U.cpu().numpy()
    assert oracle.rel_l2(u, ref) <= 1e-6
    assert np.max(np.abs(u[:10] - ref[:10])) <= 1e-6 * np.max(np.abs(ref))


def test_evaluate_sources_at_targets_fp32():
    """rpy_evaluate in the FP32 precision form at 3 digits, targets on and near sources."""
    rng = np.random.default_rng(43)
    src = synth.uniform_cube(20000, seed=44, a=0.002)
    tgt = rng.random((2000, 3))
    tgt[:5] = src.pos[:5]
    tgt[5:10] = src.pos[5:10] + 0.0007
    import torch
    U = torch.empty((len(tgt), 3), dtype=torch.float64, device="cuda")
    rp.rpy_evaluate(cuda_tensor(src.pos), cuda_tensor(src.f), cuda_tensor(tgt), src.a, src.s, 3, U,
                    precision=rp.RPY_FP32)
    pos = np.concatenate([src.pos, tgt])
    f = np.concatenate([src.f, np.zeros_like(tgt)])
    ref = oracle.rpy_direct(pos, f, src.a, src.s, targets=np.arange(src.n, src.n + len(tgt)))
    assert oracle.rel_l2(U.cpu().numpy(), ref) <= 1e-3


def test_autotune_verifies_its_choice_on_a_fresh_deep_sample():
    """With the loosest search margin (accept a sampled error up to the bound itself on
    64 targets), the tuner's choice must still pass its verification: an independent
    FP64 direct sum on 256 fresh targets, half in the two deepest leaf levels, at half
    the bound.  The verified choice meets the setting against the oracle."""
    sysm = synth.sphere_plus_cube(200000, seed=33, a=1e-4)
    P, F = cuda_tensor(sysm.pos), cuda_tensor(sysm.f)
    res = rp.rpy_autotune(P, [0, sysm.n], [sysm.a], F, sysm.s, 6, rp.RPY_FP32, n_samples=64, timed_reps=1,
                          margin=1.0)
    best = res["best"]
    assert res["n_verify"] == 256
    assert res["verify_ok"] and res["verify_rel_l2"] <= 0.5e-6
    assert best["precision"] in (rp.RPY_FP32, rp.RPY_FP64)
    import torch
    t = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 6, leaf_cap=best["leaf_cap"], precision=best["precision"],
                            order_p=best["order_p"], direct_w=best["direct_w"], direct_x=best["direct_x"],
                            quad=best["quad"])
    U = torch.empty_like(F)
    rp.rpy_forest_matvec(t, F, [sysm.s], U)
    rp.rpy_tree_sync(t)
    tg = synth.sample_targets(sysm.n, k=400, seed=78)
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg)
    assert oracle.rel_l2(U.cpu().numpy()[tg], ref) <= 1e-6
    t.close()
