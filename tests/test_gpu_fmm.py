"""GPU parity of the RPY matvec against the CPU oracle, through the C ABI.

Tolerances: the permutation and the Morton keys are bit-exact; the direct
(single-leaf) path and the near part agree with the oracle to 1e-12 relative
(FP64 rounding of ~N terms); the FMM meets its digit setting, rel-L2 <= 1e-3
(3 digits) or <= 1e-6 (6 digits), on the full velocity and on the far part
alone (velocity minus near part).
"""
import math

import numpy as np
import pytest

import oracle
import paper_1711_02976_gb300 as rp
import synth
from gpu_util import box_members, csr, cuda_tensor, leaf_members, matvec

pytestmark = pytest.mark.gpu


def _near_oracle(t, pos, f, a, s):
    """Oracle restricted to the U list of every leaf (self term included)."""
    lm = leaf_members(t)
    leaves = rp.rpy_tree_export(t, "leaves")
    ul = csr(t, "u_off", "u_idx")
    out = np.zeros_like(f)
    for li, b in enumerate(leaves):
        tg = lm[int(b)]
        src = np.concatenate([lm[int(c)] for c in ul[li]])
        # put the targets first so that the oracle's index i matches
        rest = np.setdiff1d(src, tg)
        idx = np.concatenate([tg, rest])
        out[tg] = oracle.rpy_direct(pos[idx], f[idx], a, s, targets=np.arange(len(tg)))
    return out


# ---------------------------------------------------------------- tree

def test_permutation_and_keys_bit_exact():
    sysm = synth.config1()
    P = cuda_tensor(sysm.pos)
    t = rp.rpy_tree_build(P, sysm.n, sysm.a, 3, leaf_cap=40)
    keys, cube = oracle.morton_keys(sysm.pos)
    perm = oracle.stable_sort(keys)
    np.testing.assert_array_equal(rp.rpy_tree_export(t, "perm"), perm)
    np.testing.assert_array_equal(rp.rpy_tree_export(t, "keys"), keys[perm])
    np.testing.assert_array_equal(rp.rpy_tree_export(t, "cube")[0], cube)


def test_morton_keys_exact_on_and_near_grid_points():
    """Coordinates whose scaled value (x - origin) / side * 2^21 is an integer (a cube of side 1
    and coordinates on a 2^-12 grid), or lies within rounding of one (a cube of side 3, offsets of
    0, 1e-12 and 3e-10 key cells): the key kernel's multiply-by-reciprocal path must defer to the
    correctly rounded division there.  Keys and order bit-exact against the oracle."""
    rng = np.random.default_rng(12)
    n = 20000
    on_grid = rng.integers(0, 4097, size=(n, 3)) / 4096.0
    on_grid[0], on_grid[1] = 0.0, 1.0
    k = rng.integers(0, 2 ** 21, size=(n, 3)).astype(np.float64)
    delta = rng.choice([-3e-10, -1e-12, 0.0, 1e-12, 3e-10], size=(n, 3))
    near_grid = 3.0 * (k + delta) / 2 ** 21
    near_grid[0], near_grid[1] = 0.0, 3.0
    for pos in (on_grid, near_grid):
        t = rp.rpy_tree_build(cuda_tensor(pos), n, 1e-6, 3, leaf_cap=40)
        keys, cube = oracle.morton_keys(pos)
        perm = oracle.stable_sort(keys)
        np.testing.assert_array_equal(rp.rpy_tree_export(t, "keys"), keys[perm])
        np.testing.assert_array_equal(rp.rpy_tree_export(t, "perm"), perm)
        np.testing.assert_array_equal(rp.rpy_tree_export(t, "cube")[0], cube)


def test_forest_permutation_bit_exact():
    rng = np.random.default_rng(5)
    sizes = [1, 700, 33, 2000]
    pos = [rng.random((n, 3)) * (k + 1) for k, n in enumerate(sizes)]
    pos[2][:] = pos[2][0]                      # a degenerate system (all beads at one point)
    off = np.concatenate([[0], np.cumsum(sizes)])
    t = rp.rpy_forest_build(cuda_tensor(np.concatenate(pos)), off, [0.01] * 4, 3, leaf_cap=16)
    got = rp.rpy_tree_export(t, "perm")
    for k in range(4):
        keys, _ = oracle.morton_keys(pos[k])
        np.testing.assert_array_equal(got[off[k]:off[k + 1]], off[k] + oracle.stable_sort(keys))


def _clustered(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((n // 2, 3))
    b = 0.5 + 0.03 * rng.standard_normal((n - n // 2, 3))
    return np.concatenate([a, b])


@pytest.mark.parametrize("direct", [(-1, -1), (0, 0), (20, 30)])
def test_tree_invariants_and_list_coverage(direct):
    """Every bead is in exactly one leaf; the U, V, W, X lists and the direct
    substitutes of small W / X interactions cover every ordered pair of beads
    exactly once (brute force)."""
    pos = _clustered(1500, 1)
    t = rp.rpy_forest_build(cuda_tensor(pos), [0, len(pos)], [1e-4], 3, leaf_cap=6, direct_w=direct[0],
                            direct_x=direct[1])
    n = len(pos)
    lm = leaf_members(t)
    allm = np.concatenate(list(lm.values()))
    assert np.array_equal(np.sort(allm), np.arange(n))
    st = rp.rpy_tree_stats(t)
    assert st["max_leaf_count"] <= 6 and st["n_leaves"] == len(lm)
    bm = box_members(t)
    leaves = rp.rpy_tree_export(t, "leaves")
    U, W = csr(t, "u_off", "u_idx"), csr(t, "w_off", "w_idx")
    V, X = csr(t, "v_off", "v_idx"), csr(t, "x_off", "x_idx")
    Dl = csr(t, "d_off", "d_idx")
    nw, nx, nd = (sum(len(z) for z in L) for L in (W, X, Dl))
    if direct[0] < 0:
        assert nd == 0 and nw > 0 and nx > 0          # the tree is adaptive
    else:
        assert nd > 0
    cnt = np.zeros((n, n), dtype=np.int32)
    for li, b in enumerate(leaves):
        for c in U[li]:
            cnt[np.ix_(bm[b], bm[c])] += 1
        for c in W[li]:
            cnt[np.ix_(bm[b], bm[c])] += 1
        for c in Dl[li]:
            cnt[np.ix_(bm[b], bm[c])] += 1
    for b in range(len(bm)):
        for c in V[b]:
            cnt[np.ix_(bm[b], bm[c])] += 1
        for c in X[b]:
            cnt[np.ix_(bm[b], bm[c])] += 1
    assert cnt.min() == 1 and cnt.max() == 1
    # lists are symmetric where the definitions say so
    if direct[0] < 0:
        for li, b in enumerate(leaves):
            for c in W[li]:
                assert b in X[c]
    for li, b in enumerate(leaves):
        assert b in U[li]


# ---------------------------------------------------------------- direct parity

def test_single_leaf_equals_direct_sum():
    rng = np.random.default_rng(2)
    n = 1000
    pos = rng.random((n, 3)) * 0.2
    f = rng.standard_normal((n, 3))
    a = 0.01                                   # many overlapping pairs
    pos[7] = pos[8]                            # one coincident pair
    s = 6 * math.pi * a
    u, t = matvec(pos, f, a, s, 3, leaf_cap=n)
    assert rp.rpy_tree_stats(t)["n_leaves"] == 1
    ref = oracle.rpy_direct(pos, f, a, s)
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()


def test_near_part_matches_oracle_on_u_lists():
    sysm = synth.config1()
    u, t = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3, leaf_cap=40, parts=rp.RPY_PART_NEAR)
    ref = _near_oracle(t, sysm.pos, sysm.f, sysm.a, sysm.s)
    assert np.abs(u - ref).max() < 1e-12 * np.abs(ref).max()


def _close_pairs(n, a, seed):
    """Uniform beads plus partners closer than 2a: 300 in (0, 2a), 20 within 1e-4 a,
    10 coincident."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * 0.9 + 0.05
    k = 0
    for cnt, lo, hi in ((300, 0.0, 2.0 * a), (20, 0.0, 1e-4 * a), (10, 0.0, 0.0)):
        for _ in range(cnt):
            d = rng.standard_normal(3)
            pos[n - 1 - k] = pos[k] + (lo + (hi - lo) * rng.random()) * d / np.linalg.norm(d)
            k += 1
    return pos, rng.standard_normal((n, 3))


@pytest.mark.parametrize("a", [0.002, 0.01])   # leaves ~60a and ~12a wide
def test_fp32_near_part_matches_oracle_on_u_lists(a):
    """FP32 near field (compensated FP32 sums, FP64 for pairs within 1e-3 a)
    against the oracle on the U lists, with many overlapping, nearly coincident
    and coincident pairs."""
    pos, f = _close_pairs(6000, a, 71)
    s = 6 * math.pi * a
    u, t = matvec(pos, f, a, s, 3, leaf_cap=40, precision=rp.RPY_FP32, parts=rp.RPY_PART_NEAR)
    ref = _near_oracle(t, pos, f, a, s)
    assert np.abs(u - ref).max() < 2e-6 * np.abs(ref).max()


def test_fp32_close_pairs_beyond_the_queue():
    """A cluster of 48 beads within 1e-4 a of one point (a quarter of them coincident) sits in
    one leaf (the 2a rule stops refinement there): 2,256 ordered pairs closer than 1e-3 a meet
    in one staged chunk, more than the near-field kernel's shared-memory queue holds, so every
    thread re-scans its sources for them in FP64.  The FP32 near part still matches the oracle."""
    rng = np.random.default_rng(17)
    n, a = 3000, 0.002
    pos = rng.random((n, 3)) * 0.9 + 0.05
    c0 = pos[0].copy()
    for k in range(1, 48):
        d = rng.standard_normal(3)
        pos[k] = c0 if k % 4 == 0 else c0 + 1e-4 * a * rng.random() * d / np.linalg.norm(d)
    f = rng.standard_normal((n, 3))
    s = 6 * math.pi * a
    u, t = matvec(pos, f, a, s, 3, leaf_cap=40, precision=rp.RPY_FP32, parts=rp.RPY_PART_NEAR)
    assert rp.rpy_tree_stats(t)["max_leaf_count"] >= 48
    ref = _near_oracle(t, pos, f, a, s)
    assert np.abs(u - ref).max() < 2e-6 * np.abs(ref).max()
    # the cluster's beads themselves (their sums are dominated by the close pairs)
    np.testing.assert_allclose(u[:48], ref[:48], rtol=0, atol=2e-6 * np.abs(ref[:48]).max())


# ---------------------------------------------------------------- far field operators

@pytest.mark.parametrize("digits,tol", [(3, 1e-3), (6, 1e-6), (9, 1e-9)])
def test_laplace_far_field_against_direct_sums(digits, tol):
    """Potential, gradient and Hessian of the four Laplace sets from the FMM
    (everything outside each leaf's U list) against direct sums.  The digit
    setting bounds the potential; each derivative multiplies the truncation
    error of an order-p expansion by roughly (p+1)/(separation), so the
    gradient is held to 3x and the Hessian to 10x the setting at p <= 18, and
    to 10x and 200x at the 9-digit order p = 26 (measured: Hessian 7.8e-8)."""
    import torch
    pos = _clustered(3000, 3)
    rng = np.random.default_rng(4)
    q = rng.standard_normal((len(pos), 4))
    # pure FMM: every W interaction by multipole evaluation (Theorem 1), every X by P2L
    t = rp.rpy_forest_build(cuda_tensor(pos), [0, len(pos)], [1e-5], digits, leaf_cap=12, direct_w=-1, direct_x=-1)
    assert rp.rpy_tree_stats(t)["n_wlist"] > 0
    out = torch.empty((len(pos), 4, 13), dtype=torch.float64, device="cuda")
    rp.rpy_laplace_far(t, cuda_tensor(q), out)
    got = out.cpu().numpy()
    lm = leaf_members(t)
    leaves = rp.rpy_tree_export(t, "leaves")
    ul = csr(t, "u_off", "u_idx")
    ref = np.zeros_like(got)
    for li, b in enumerate(leaves):
        tg = lm[int(b)]
        near = np.concatenate([lm[int(c)] for c in ul[li]])
        far = np.setdiff1d(np.arange(len(pos)), near)
        if len(far) == 0:
            continue
        phi, g, H = oracle.laplace_direct(pos[far], q[far], pos[tg])
        ref[tg, :, 0] = phi
        ref[tg, :, 1:4] = g
        ref[tg, :, 4:13] = H.reshape(len(tg), 4, 9)
    fg, fh = (10, 200) if digits == 9 else (3, 10)
    for name, sl, f in (("phi", slice(0, 1), 1), ("grad", slice(1, 4), fg), ("hess", slice(4, 13), fh)):
        e = oracle.rel_l2(got[:, :, sl], ref[:, :, sl])
        assert e < f * tol, (name, e)


# ---------------------------------------------------------------- full matvec parity

def _check(pos, f, a, s, digits, tol, targets=None, **kw):
    u, t = matvec(pos, f, a, s, digits, **kw)
    if targets is None:
        ref = oracle.rpy_direct(pos, f, a, s)
        uu = u
    else:
        ref = oracle.rpy_direct(pos, f, a, s, targets=targets)
        uu = u[targets]
    fi = f if targets is None else f[targets]
    self_t = s / (6 * math.pi * a) * fi
    e = oracle.rel_l2(uu, ref)
    e_far = oracle.rel_l2(uu - self_t, ref - self_t)
    assert e < tol, e
    assert e_far < 5 * tol, e_far
    return e, e_far, t


@pytest.mark.parametrize("digits,tol", [(3, 1e-3), (6, 1e-6), (9, 1e-9)])
def test_config1_parity(digits, tol):
    sysm = synth.config1()
    _check(sysm.pos, sysm.f, sysm.a, sysm.s, digits, tol, leaf_cap=40)


@pytest.mark.parametrize("digits,tol", [(3, 1e-3), (6, 1e-6), (9, 1e-9)])
def test_direct_substitution_matches_pure_fmm(digits, tol):
    """Small W / X interactions summed directly give the same velocity as the
    multipole / local expansions they replace, both within the setting."""
    sysm = synth.sphere_plus_cube(30000, 21, 1e-4)
    tg = synth.sample_targets(sysm.n, 600)
    e0, _, t0 = _check(sysm.pos, sysm.f, sysm.a, sysm.s, digits, tol, targets=tg, leaf_cap=40, direct_w=-1,
                       direct_x=-1)
    e1, _, t1 = _check(sysm.pos, sysm.f, sysm.a, sysm.s, digits, tol, targets=tg, leaf_cap=40)
    s0, s1 = rp.rpy_tree_stats(t0), rp.rpy_tree_stats(t1)
    assert s0["n_dlist"] == 0 and s0["n_wlist"] > 0
    assert s1["n_dlist"] > 0 and s1["n_wlist"] < s0["n_wlist"]


def test_dipole_term_regime():
    """a comparable to the box size, where the a^2/r^2 (grad L_C) term is large:
    a wrong sign of the dipole term would fail here."""
    rng = np.random.default_rng(6)
    pos = rng.random((512, 3))
    f = rng.standard_normal((512, 3))
    a = 0.02
    e, e_far, t = _check(pos, f, a, 6 * math.pi * a, 6, 1e-6, leaf_cap=8)
    assert rp.rpy_tree_stats(t)["depth"] >= 2


def test_adaptive_sphere_6digit():
    sysm = synth.sphere_plus_cube(20000, 12, 2e-4)
    tg = synth.sample_targets(sysm.n, 1000)
    _check(sysm.pos, sysm.f, sysm.a, sysm.s, 6, 1e-6, targets=tg, leaf_cap=30)


def test_bench_configuration_sampled_parity():
    """The benchmark workload (1M beads, sphere surface + 10% cube, a = 1e-4,
    6 digits, FP64) on 2,000 sampled targets."""
    sysm = synth.config2()
    tg = synth.sample_targets(sysm.n)
    _check(sysm.pos, sysm.f, sysm.a, sysm.s, 6, 1e-6, targets=tg)


def test_fp32_precision_form_3digit():
    sysm = synth.config1()
    _check(sysm.pos, sysm.f, sysm.a, sysm.s, 3, 1e-3, leaf_cap=40, precision=rp.RPY_FP32)


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("precision", [rp.RPY_FP64, rp.RPY_FP32])
def test_single_bead(precision):
    u, t = matvec(np.array([[0.2, 0.3, 0.4]]), np.array([[1.0, -2.0, 0.5]]), 0.1, 2.0, 3, precision=precision)
    np.testing.assert_allclose(u, 2.0 / (6 * math.pi * 0.1) * np.array([[1.0, -2.0, 0.5]]), rtol=1e-15)


@pytest.mark.parametrize("precision,tol", [(rp.RPY_FP64, 1e-12), (rp.RPY_FP32, 1e-6)])
def test_all_beads_coincident(precision, tol):
    """50 beads at one point: every pair is the r -> 0 limit.  In the FP32 form all 2,450 of
    them are taken in FP64, beyond the near-field kernel's shared-memory queue."""
    pos = np.tile([[0.5, 0.5, 0.5]], (50, 1))
    f = np.random.default_rng(0).standard_normal((50, 3))
    u, t = matvec(pos, f, 0.1, 1.0, 3, leaf_cap=4, precision=precision)
    ref = oracle.rpy_direct(pos, f, 0.1, 1.0)
    assert np.abs(u - ref).max() < tol * np.abs(ref).max()


@pytest.mark.parametrize("precision", [rp.RPY_FP64, rp.RPY_FP32])
def test_ragged_sizes_and_tiny_leaves(precision):
    rng = np.random.default_rng(8)
    for n in (2, 3, 129, 4097):
        pos = rng.random((n, 3))
        f = rng.standard_normal((n, 3))
        a = 0.001
        u, t = matvec(pos, f, a, 6 * math.pi * a, 3, leaf_cap=3, precision=precision)
        ref = oracle.rpy_direct(pos, f, a, 6 * math.pi * a)
        assert oracle.rel_l2(u, ref) < 1e-3, n


def test_overlap_rule_stops_refinement():
    """Beads closer than 2a are never split apart: leaves may exceed the cap."""
    rng = np.random.default_rng(9)
    pos = 0.5 + 0.002 * rng.standard_normal((400, 3))
    f = rng.standard_normal((400, 3))
    a = 0.01
    u, t = matvec(pos, f, a, 6 * math.pi * a, 3, leaf_cap=5)
    st = rp.rpy_tree_stats(t)
    assert st["leaves_over_cap"] >= 1
    side = rp.rpy_tree_export(t, "box_side")
    assert side.min() >= 2 * a or st["n_boxes"] == 1
    ref = oracle.rpy_direct(pos, f, a, 6 * math.pi * a)
    assert oracle.rel_l2(u, ref) < 1e-12


def test_nonfinite_and_invalid_inputs():
    import torch
    pos = np.random.default_rng(0).random((100, 3))
    pos[17, 1] = np.nan
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_tree_build(cuda_tensor(pos), 100, 0.01, 3)
    assert e.value.status == -6
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_tree_build(cuda_tensor(pos), 100, 0.0, 3)
    assert e.value.status == -1
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_tree_build(cuda_tensor(pos), 100, 0.01, 5)
    assert e.value.status == -2


def test_translation_and_linearity():
    sysm = synth.config1()
    u0, _ = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3)
    u1, _ = matvec(sysm.pos + np.array([1e3, -1e3, 1e3]), sysm.f, sysm.a, sysm.s, 3)
    assert oracle.rel_l2(u1, u0) < 1e-6
    u2, _ = matvec(sysm.pos, 2.0 * sysm.f, sysm.a, 3.0 * sysm.s, 3)
    assert oracle.rel_l2(u2, 6.0 * u0) < 1e-13


def test_forest_results_equal_individual_systems():
    import torch
    rng = np.random.default_rng(11)
    sizes = [3000, 500, 1200]
    pos = [rng.random((n, 3)) for n in sizes]
    f = [rng.standard_normal((n, 3)) for n in sizes]
    a = [0.004, 0.01, 0.002]
    s = [1.0, 2.0, 0.5]
    off = np.concatenate([[0], np.cumsum(sizes)])
    F = cuda_tensor(np.concatenate(f))
    U = torch.empty_like(F)
    t = rp.rpy_forest_build(cuda_tensor(np.concatenate(pos)), off, a, 3, leaf_cap=20)
    rp.rpy_forest_matvec(t, F, s, U)
    got = U.cpu().numpy()
    for k in range(3):
        uk, _ = matvec(pos[k], f[k], a[k], s[k], 3, leaf_cap=20)
        np.testing.assert_array_equal(got[off[k]:off[k + 1]], uk)


@pytest.mark.parametrize("precision,digits,tol", [(rp.RPY_FP64, 6, 1e-6), (rp.RPY_FP32, 3, 1e-3)])
def test_forest_with_degenerate_systems(precision, digits, tol):
    """One forest of degenerate systems beside ordinary ones: a single bead (a cube of side 0),
    two coincident beads, two beads far apart, three beads within 2a of each other, a system whose
    beads all sit on one plane (a cube flat on one axis), and a 6,000-bead cube deep enough for a
    far field.  Every system against the oracle on its own, in both precision forms."""
    import torch
    rng = np.random.default_rng(21)
    plane = rng.random((400, 3))
    plane[:, 2] = 0.25
    systems = [
        (np.array([[0.3, 0.4, 0.5]]), 0.01),
        (np.array([[0.2, 0.2, 0.2], [0.2, 0.2, 0.2]]), 0.01),
        (np.array([[0.0, 0.0, 0.0], [10.0, -3.0, 2.0]]), 0.01),
        (np.array([[0.5, 0.5, 0.5], [0.505, 0.5, 0.5], [0.5, 0.508, 0.5]]), 0.01),
        (plane, 0.004),
        (rng.random((6000, 3)), 0.002),
    ]
    pos = [sy[0] for sy in systems]
    a = [sy[1] for sy in systems]
    s = [6 * math.pi * ak for ak in a]
    f = [rng.standard_normal(p_.shape) for p_ in pos]
    off = np.concatenate([[0], np.cumsum([len(p_) for p_ in pos])]).astype(np.int64)
    t = rp.rpy_forest_build(cuda_tensor(np.concatenate(pos)), off, a, digits, leaf_cap=20, precision=precision)
    U = torch.empty((int(off[-1]), 3), dtype=torch.float64, device="cuda")
    rp.rpy_forest_matvec(t, cuda_tensor(np.concatenate(f)), s, U)
    rp.rpy_tree_sync(t)
    u = U.cpu().numpy()
    assert rp.rpy_tree_stats(t)["depth"] >= 3
    for k in range(len(systems)):
        ref = oracle.rpy_direct(pos[k], f[k], a[k], s[k])
        assert oracle.rel_l2(u[off[k]:off[k + 1]], ref) <= tol, k


def _forest_parity(systems, digits, tol, **kw):
    import torch
    pos = [sy[0] for sy in systems]
    a = [sy[1] for sy in systems]
    s = [6 * math.pi * ak for ak in a]
    rng = np.random.default_rng(33)
    f = [rng.standard_normal(p_.shape) for p_ in pos]
    off = np.concatenate([[0], np.cumsum([len(p_) for p_ in pos])]).astype(np.int64)
    t = rp.rpy_forest_build(cuda_tensor(np.concatenate(pos)), off, a, digits, **kw)
    U = torch.empty((int(off[-1]), 3), dtype=torch.float64, device="cuda")
    rp.rpy_forest_matvec(t, cuda_tensor(np.concatenate(f)), s, U)
    rp.rpy_tree_sync(t)
    u = U.cpu().numpy()
    for k in range(len(systems)):
        tg = synth.sample_targets(len(pos[k]), 300, seed=40 + k)
        ref = oracle.rpy_direct(pos[k], f[k], a[k], s[k], targets=tg)
        assert oracle.rel_l2(u[off[k] + tg], ref) <= tol, k
    return t


@pytest.mark.parametrize("precision", [rp.RPY_FP64, rp.RPY_FP32])
def test_cartesian_far_field_on_a_forest(precision):
    """The polynomial far field with several systems in one tree (each its own cube, its own
    boxes and V lists): a uniform cube, a sphere surface and a clustered system of different
    sizes and radii, every one against the oracle at 3 digits."""
    rng = np.random.default_rng(34)
    systems = [(rng.random((12000, 3)), 0.002),
               (synth._sphere_surface(rng, 8000, 0.5, (0.5, 0.5, 0.5)), 0.001),
               (_clustered(6000, 35) * 3.0, 0.003)]
    t = _forest_parity(systems, 3, 1e-3, leaf_cap=40, precision=precision, flags=rp.RPY_FLAG_CARTESIAN)
    assert rp.rpy_tree_stats(t)["depth"] >= 3


def test_9digit_forest():
    """Nine digits (FP64) with two systems of different scales in one tree."""
    rng = np.random.default_rng(36)
    systems = [(rng.random((8000, 3)), 0.002),
               (synth._sphere_surface(rng, 6000, 2.0, (1.0, -1.0, 0.5)), 0.004)]
    _forest_parity(systems, 9, 1e-9, leaf_cap=60)


def test_host_entry_point():
    sysm = synth.config1()
    u = np.zeros_like(sysm.f)
    rp.rpy_matvec_host(np.ascontiguousarray(sysm.pos), sysm.a, np.ascontiguousarray(sysm.f), sysm.s, 3, u)
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s)
    assert oracle.rel_l2(u, ref) < 1e-3


def test_resident_tree_host_buffer_matvec():
    """rpy_tree_matvec_host (host arrays in and out on a resident tree) gives the device-
    pointer path's velocities bitwise: with new positions (rebuild inside the call), with
    positions unchanged (pos NULL), and with pageable as well as page-locked buffers."""
    import torch
    sysm = synth.sphere_plus_cube(20000, 61, 2e-4)
    t = rp.rpy_tree_build(cuda_tensor(sysm.pos), sysm.n, sysm.a, 6)
    pos2 = np.ascontiguousarray(sysm.pos + 1e-3 * np.random.default_rng(2).standard_normal(sysm.pos.shape))
    f = np.ascontiguousarray(sysm.f)
    u = np.zeros_like(f)
    rp.rpy_tree_matvec_host(t, pos2, f, sysm.s, u)
    ref, _ = matvec(pos2, sysm.f, sysm.a, sysm.s, 6)
    np.testing.assert_array_equal(u, ref)
    f2 = torch.from_numpy(-2.0 * f).pin_memory().numpy()
    u2 = torch.zeros(f.shape, dtype=torch.float64).pin_memory().numpy()
    rp.rpy_tree_matvec_host(t, None, f2, sysm.s, u2)
    np.testing.assert_array_equal(u2, -2.0 * ref)   # the matvec is linear, and -2x is exact
    # new positions and forces from page-locked buffers (the forces' copy then runs
    # asynchronously beside the rebuild), twice in a row
    pos3 = torch.from_numpy(np.ascontiguousarray(sysm.pos[::-1] * 0.9 + 0.05)).pin_memory().numpy()
    f3 = torch.from_numpy(np.ascontiguousarray(f[::-1])).pin_memory().numpy()
    for _ in range(2):
        u3 = torch.zeros(f.shape, dtype=torch.float64).pin_memory().numpy()
        rp.rpy_tree_matvec_host(t, pos3, f3, sysm.s, u3)
        ref3, _ = matvec(pos3, f3, sysm.a, sysm.s, 6)
        np.testing.assert_array_equal(u3, ref3)
    tg = synth.sample_targets(sysm.n, 500)
    assert oracle.rel_l2(u[tg], oracle.rpy_direct(pos2, f, sysm.a, sysm.s, targets=tg)) < 1e-6
    t.close()


def test_update_positions_matches_fresh_build():
    import torch
    sysm = synth.config1()
    P = cuda_tensor(sysm.pos)
    F = cuda_tensor(sysm.f)
    t = rp.rpy_tree_build(P, sysm.n, sysm.a, 3)
    pos2 = sysm.pos + 1e-3 * np.random.default_rng(1).standard_normal(sysm.pos.shape)
    rp.rpy_tree_update_positions(t, cuda_tensor(pos2))
    U = torch.empty_like(F)
    rp.rpy_matvec(t, F, sysm.s, U)
    u2, _ = matvec(pos2, sysm.f, sysm.a, sysm.s, 3)
    np.testing.assert_array_equal(U.cpu().numpy(), u2)


@pytest.mark.parametrize("precision", [rp.RPY_FP64, rp.RPY_FP32])
def test_forest_update_positions_matches_fresh_build(precision):
    """A forest rebuilt in place for new positions (as each Brownian-dynamics step does) gives
    bitwise the velocities of a forest built fresh at those positions, graph replay included."""
    import torch
    rng = np.random.default_rng(37)
    sizes = [3000, 500, 9000]
    pos = [rng.random((n, 3)) * (k + 1) for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    a, s = [0.004, 0.01, 0.003], [1.0, 2.0, 0.5]
    P = np.concatenate(pos)
    F = cuda_tensor(rng.standard_normal(P.shape))
    t = rp.rpy_forest_build(cuda_tensor(P), off, a, 3, leaf_cap=30, precision=precision)
    U = torch.empty_like(F)
    for _ in range(2):
        rp.rpy_forest_matvec(t, F, s, U)   # the second replays the captured graph
    P2 = P + 1e-3 * rng.standard_normal(P.shape)
    rp.rpy_tree_update_positions(t, cuda_tensor(P2))
    for _ in range(2):
        rp.rpy_forest_matvec(t, F, s, U)
    t2 = rp.rpy_forest_build(cuda_tensor(P2), off, a, 3, leaf_cap=30, precision=precision)
    U2 = torch.empty_like(F)
    rp.rpy_forest_matvec(t2, F, s, U2)
    rp.rpy_tree_sync(t2)
    np.testing.assert_array_equal(U.cpu().numpy(), U2.cpu().numpy())


def test_graph_replay_matches_plain_launches():
    """From the second matvec on a build, the body runs as a captured CUDA graph;
    results stay bitwise equal to plain launches, also after a rebuild."""
    import torch
    sysm = synth.sphere_plus_cube(20000, 31, 2e-4)
    P, F = cuda_tensor(sysm.pos), cuda_tensor(sysm.f)
    t_graph = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 6, leaf_cap=40)
    t_plain = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 6, leaf_cap=40, flags=1)
    U0, U1 = torch.empty_like(F), torch.empty_like(F)
    for rep in range(3):
        rp.rpy_matvec(t_graph, F, sysm.s, U0)
        rp.rpy_matvec(t_plain, F, sysm.s, U1)
        torch.cuda.synchronize()
        assert torch.equal(U0, U1), rep
    P2 = cuda_tensor(sysm.pos + 1e-4 * np.random.default_rng(0).standard_normal(sysm.pos.shape))
    rp.rpy_tree_update_positions(t_graph, P2)
    rp.rpy_tree_update_positions(t_plain, P2)
    for rep in range(3):
        rp.rpy_matvec(t_graph, 2.0 * F, sysm.s, U0)
        rp.rpy_matvec(t_plain, 2.0 * F, sysm.s, U1)
        torch.cuda.synchronize()
        assert torch.equal(U0, U1), rep


def test_matvec_batched_equals_separate_calls():
    import torch
    A = synth.uniform_cube(5000, seed=51, a=0.003)
    B = synth.sphere_plus_cube(7000, seed=52, a=0.002)
    ta = rp.rpy_tree_build(cuda_tensor(A.pos), A.n, A.a, 6)
    tb = rp.rpy_tree_build(cuda_tensor(B.pos), B.n, B.a, 3)
    Fa, Fb = cuda_tensor(A.f), cuda_tensor(B.f)
    Ua, Ub = torch.empty_like(Fa), torch.empty_like(Fb)
    rp.rpy_matvec_batched([ta, tb], [Fa, Fb], [A.s, 2.0 * B.s], [Ua, Ub])
    Va, Vb = torch.empty_like(Fa), torch.empty_like(Fb)
    rp.rpy_matvec(ta, Fa, A.s, Va)
    rp.rpy_matvec(tb, Fb, 2.0 * B.s, Vb)
    torch.cuda.synchronize()
    assert torch.equal(Ua, Va) and torch.equal(Ub, Vb)


@pytest.mark.parametrize("precision,digits", [(rp.RPY_FP64, 6), (rp.RPY_FP32, 3)])
def test_one_frame_per_pass_matches_all_frames(precision, digits):
    """RPY_FLAG_FRAME_PASSES (M2X / X2X / X2L one plane-wave frame at a time, the
    layout of trees too large for the six-direction buffers) gives the result of
    the single pass up to the order in which the three frames' local expansions
    are added, and meets the digit setting against the oracle."""
    import torch
    sysm = synth.sphere_plus_cube(20000, 61, 2e-4)
    P, F = cuda_tensor(sysm.pos), cuda_tensor(sysm.f)
    U0, U1 = torch.empty_like(F), torch.empty_like(F)
    t0 = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], digits, leaf_cap=30, precision=precision)
    t1 = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], digits, leaf_cap=30, precision=precision,
                             flags=rp.RPY_FLAG_FRAME_PASSES)
    assert rp.rpy_tree_stats(t1)["device_bytes"] < rp.rpy_tree_stats(t0)["device_bytes"]
    for rep in range(2):   # plain launches, then the captured graph
        rp.rpy_matvec(t0, F, sysm.s, U0)
        rp.rpy_matvec(t1, F, sysm.s, U1)
        torch.cuda.synchronize()
        u0, u1 = U0.cpu().numpy(), U1.cpu().numpy()
        tol = 1e-13 if precision == rp.RPY_FP64 else 1e-6
        assert np.max(np.abs(u1 - u0)) <= tol * np.max(np.abs(u0)), rep
    tg = synth.sample_targets(sysm.n, 500)
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg)
    assert oracle.rel_l2(u1[tg], ref) <= (1e-6 if digits == 6 else 1e-3)


@pytest.mark.parametrize("precision,digits", [(rp.RPY_FP64, 6), (rp.RPY_FP32, 3)])
def test_per_component_evaluation_equals_per_potential(precision, digits):
    """Approach 2 of Sec. 2 (the default: six expansions per bead, u_d = H_d -
    |x|^2 B_d) against approach 1 (RPY_FLAG_EVAL_PER_POTENTIAL: folded values and
    nine gradients per bead): the same far field up to rounding."""
    import torch
    sysm = synth.sphere_plus_cube(20000, 63, 2e-4)
    P, F = cuda_tensor(sysm.pos), cuda_tensor(sysm.f)
    U2, U1 = torch.empty_like(F), torch.empty_like(F)
    t2 = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], digits, leaf_cap=30, precision=precision)
    t1 = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], digits, leaf_cap=30, precision=precision,
                             flags=rp.RPY_FLAG_EVAL_PER_POTENTIAL)
    rp.rpy_matvec_parts(t2, F, sysm.s, U2, rp.RPY_PART_FAR)
    rp.rpy_matvec_parts(t1, F, sysm.s, U1, rp.RPY_PART_FAR)
    torch.cuda.synchronize()
    u2, u1 = U2.cpu().numpy(), U1.cpu().numpy()
    tol = 1e-11 if precision == rp.RPY_FP64 else 2e-5
    assert np.max(np.abs(u2 - u1)) <= tol * np.max(np.abs(u1))


def test_9digit_sphere_sampled_parity():
    """The 9-digit setting (FP64, plane-wave rule of 2.3e-10, default p = 26) on an
    adaptive 100k-bead sphere + cube against the oracle on 1,000 targets; the FP32
    form is refused at 9 digits."""
    sysm = synth.sphere_plus_cube(100000, 81, 1e-4)
    tg = synth.sample_targets(sysm.n, 1000)
    e, e_far, t = _check(sysm.pos, sysm.f, sysm.a, sysm.s, 9, 1e-9, targets=tg)
    st = rp.rpy_tree_stats(t)
    assert st["digits"] == 9 and st["order_p"] == 26 and st["quad"] in (0, 9)
    with pytest.raises(Exception):
        rp.rpy_forest_build(cuda_tensor(sysm.pos), [0, sysm.n], [sysm.a], 9, precision=rp.RPY_FP32)


def test_laplace_far_field_error_decays_with_order_and_hessian_is_traceless():
    """The Laplace far field of the FMM (9-digit plane-wave rule, so that the
    truncation at order p dominates; pure FMM) against direct sums at p = 4, 8, 12,
    16: the error falls by a factor of at least 3 per step of 4 in p (geometric
    decay), and the Hessian of every expansion has zero trace (the expansions are
    harmonic)."""
    import torch
    pos = _clustered(2000, 5)
    rng = np.random.default_rng(6)
    q = rng.standard_normal((len(pos), 4))
    errs = []
    for p in (4, 8, 12, 16):
        t = rp.rpy_forest_build(cuda_tensor(pos), [0, len(pos)], [1e-5], 9, leaf_cap=12, order_p=p, direct_w=-1,
                                direct_x=-1)
        out = torch.empty((len(pos), 4, 13), dtype=torch.float64, device="cuda")
        rp.rpy_laplace_far(t, cuda_tensor(q), out)
        got = out.cpu().numpy()
        lm = leaf_members(t)
        leaves = rp.rpy_tree_export(t, "leaves")
        ul = csr(t, "u_off", "u_idx")
        ref = np.zeros(got.shape[:2])
        for li, b in enumerate(leaves):
            tg = lm[int(b)]
            near = np.concatenate([lm[int(c)] for c in ul[li]])
            far = np.setdiff1d(np.arange(len(pos)), near)
            if len(far):
                ref[tg] = oracle.laplace_direct(pos[far], q[far], pos[tg])[0]
        errs.append(oracle.rel_l2(got[:, :, 0], ref))
        H = got[:, :, 4:13].reshape(len(pos), 4, 3, 3)
        assert np.abs(np.trace(H, axis1=2, axis2=3)).max() <= 1e-9 * np.abs(H).max(), p
        t.close()
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 <= e0 / 3, errs


def test_fmm_operator_is_reciprocal():
    """D is symmetric (Sec. 1, D_ij = D_ji^T): for the FMM matvec at 6 digits,
    |v.(D w) - w.(D v)| <= 1e-6 |v| |D w|."""
    import torch
    sysm = synth.sphere_plus_cube(30000, 91, 2e-4)
    rng = np.random.default_rng(92)
    v, w = rng.standard_normal((sysm.n, 3)), rng.standard_normal((sysm.n, 3))
    t = rp.rpy_tree_build(cuda_tensor(sysm.pos), sysm.n, sysm.a, 6)
    Dv, Dw = torch.empty((sysm.n, 3), dtype=torch.float64, device="cuda"), torch.empty(
        (sysm.n, 3), dtype=torch.float64, device="cuda")
    rp.rpy_matvec(t, cuda_tensor(v), sysm.s, Dv)
    rp.rpy_matvec(t, cuda_tensor(w), sysm.s, Dw)
    torch.cuda.synchronize()
    dv, dw = Dv.cpu().numpy(), Dw.cpu().numpy()
    lhs = abs(float(np.sum(v * dw)) - float(np.sum(w * dv)))
    assert lhs <= 1e-6 * np.linalg.norm(v) * np.linalg.norm(dw), lhs


@pytest.mark.parametrize("digits,tol", [(3, 2e-3), (6, 2e-6)])
def test_rotation_equivariance(digits, tol):
    """u(Q r, Q F) = Q u(r, F) for a rotation Q about the system's centre: the tree,
    the lists and the plane-wave directions all change, the velocity may not
    (beyond the digit setting)."""
    sysm = synth.sphere_plus_cube(20000, 93, 2e-4)
    rng = np.random.default_rng(94)
    A = rng.standard_normal((3, 3))
    Q, _ = np.linalg.qr(A)
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    c = np.full(3, 0.5)
    pos2 = (sysm.pos - c) @ Q.T + c
    f2 = sysm.f @ Q.T
    u1, _ = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, digits)
    u2, _ = matvec(pos2, f2, sysm.a, sysm.s, digits)
    assert oracle.rel_l2(u2, u1 @ Q.T) <= tol


def test_fp32_precision_form_6digit():
    """The FP32 form at the 6-digit setting (default p = 18: rotation-based M2M and
    L2L, FP32 plane waves) meets rel-L2 <= 1e-6 against the oracle, also as a forest."""
    sysm = synth.sphere_plus_cube(20000, 95, 2e-4)
    tg = synth.sample_targets(sysm.n, 800)
    _check(sysm.pos, sysm.f, sysm.a, sysm.s, 6, 1e-6, targets=tg, precision=rp.RPY_FP32)
    import torch
    b = synth.uniform_cube(8000, seed=96, a=0.002)
    pos = np.concatenate([sysm.pos, b.pos])
    f = np.concatenate([sysm.f, b.f])
    t = rp.rpy_forest_build(cuda_tensor(pos), [0, sysm.n, sysm.n + b.n], [sysm.a, b.a], 6,
                            precision=rp.RPY_FP32)
    U = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    rp.rpy_forest_matvec(t, cuda_tensor(f), [sysm.s, b.s], U)
    rp.rpy_tree_sync(t)
    u = U.cpu().numpy()
    ra = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s, targets=tg)
    tb = synth.sample_targets(b.n, 400)
    rb = oracle.rpy_direct(b.pos, b.f, b.a, b.s, targets=tb)
    assert oracle.rel_l2(u[tg], ra) <= 1e-6
    assert oracle.rel_l2(u[sysm.n + tb], rb) <= 1e-6


# ---------------------------------------------------------------- origin of the fourth charge set

@pytest.mark.parametrize("extra", [0, rp.RPY_FLAG_FRAME_PASSES, rp.RPY_FLAG_EVAL_PER_POTENTIAL])
@pytest.mark.parametrize("direct", [(-1, -1), (0, 0)])
def test_box_origin_equals_cube_origin_fp64(extra, direct):
    """q4 = F . (r - o) about each box's own centre, moved along with every translation
    (P2M, M2M, X2X merge and child shift, P2L, L2L, M2P and L2P re-based to the leaf), gives
    the velocity of one origin per system up to FP64 rounding: Eq. (2.8) holds for any
    common origin, and each move is the exact identity M4(o') = M4(o) + (o - o') . M_F."""
    sysm = synth.sphere_plus_cube(30000, 31, 1e-4)
    kw = dict(leaf_cap=40, direct_w=direct[0], direct_x=direct[1])
    u0, t0 = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 6, flags=rp.RPY_FLAG_CUBE_ORIGIN | extra, **kw)
    u1, t1 = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 6, flags=rp.RPY_FLAG_BOX_ORIGIN | extra, **kw)
    st = rp.rpy_tree_stats(t1)
    assert st["depth"] >= 5 and st["n_xlist"] > 0
    if direct == (-1, -1):
        assert st["n_wlist"] > 0
    assert oracle.rel_l2(u1, u0) < 1e-12


@pytest.mark.parametrize("digits,order", [(3, 8), (6, 16)])   # dense M2M / L2L below p = 12, rotations above
def test_fp32_box_origin_rounding_against_fp64(digits, order):
    """The FP32 form's rounding (its difference from the FP64 path at the same tree and
    order) with the box origin of q4 stays below the cube-origin form's on a deep adaptive
    tree, and below 0.3 x the digit setting's bound (FP32 unit roundoff is 6e-8)."""
    sysm = synth.sphere_plus_cube(400000, 41, 2e-5)
    kw = dict(order_p=order, leaf_cap=20)
    u64, t64 = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, digits, **kw)
    ub, tb = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, digits, precision=rp.RPY_FP32, flags=rp.RPY_FLAG_BOX_ORIGIN,
                    **kw)
    uc, tc = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, digits, precision=rp.RPY_FP32, flags=rp.RPY_FLAG_CUBE_ORIGIN,
                    **kw)
    assert rp.rpy_tree_stats(tb)["depth"] >= 7
    rb, rc = oracle.rel_l2(ub, u64), oracle.rel_l2(uc, u64)
    assert rb < rc, (rb, rc)
    assert rb < 0.3 * (1e-3 if digits == 3 else 1e-6), rb


@pytest.mark.parametrize("leaf_cap,depth", [(0, 7), (40, 8)])
def test_fp32_6digit_deep_sphere_2m(leaf_cap, depth):
    """The FP32 form at the 6-digit setting on a 2M-bead sphere (90% on the surface, 10%
    in the cube), at the default leaf capacity (tree depth 7) and at 40 (depth 8), against
    the oracle on 500 targets."""
    sysm = synth.sphere_plus_cube(2_000_000, 42, 1e-4)
    tg = synth.sample_targets(sysm.n, 500)
    e, e_far, t = _check(sysm.pos, sysm.f, sysm.a, sysm.s, 6, 1e-6, targets=tg, precision=rp.RPY_FP32,
                         leaf_cap=leaf_cap)
    assert rp.rpy_tree_stats(t)["depth"] >= depth


def test_batch_shaped_forest_fp32_3digit():
    """24 systems drawn like the 256-system batch (log-uniform sizes 1e3..2e5, half
    Plummer clusters, a = 0.5 / N^(1/3), so 2a is the mean spacing and the 2a rule leaves
    oversize leaves in the cluster cores), one forest, FP32 at 3 digits with default
    parameters: every system meets rel-L2 <= 1e-3 against the oracle on its own sampled
    targets, and the far part alone stays within 5x of that."""
    import torch
    systems = synth.config4(nsys=24)
    off = np.concatenate([[0], np.cumsum([sy.n for sy in systems])]).astype(np.int64)
    pos = np.concatenate([sy.pos for sy in systems])
    f = np.concatenate([sy.f for sy in systems])
    t = rp.rpy_forest_build(cuda_tensor(pos), off, [sy.a for sy in systems], 3, precision=rp.RPY_FP32)
    U = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    rp.rpy_forest_matvec(t, cuda_tensor(f), [sy.s for sy in systems], U)
    rp.rpy_tree_sync(t)
    u = U.cpu().numpy()
    st = rp.rpy_tree_stats(t)
    assert st["leaves_over_cap"] > 0   # the 2a rule binds in the cluster cores
    kinds = set()
    for k, sy in enumerate(systems):
        tg = synth.sample_targets(sy.n, 150, seed=100 + k)
        ref = oracle.rpy_direct(sy.pos, sy.f, sy.a, sy.s, targets=tg)
        got = u[off[k] + tg]
        self_t = sy.s / (6 * math.pi * sy.a) * sy.f[tg]
        assert oracle.rel_l2(got, ref) <= 1e-3, (k, sy.name)
        assert oracle.rel_l2(got - self_t, ref - self_t) <= 5e-3, (k, sy.name)
        kinds.add(sy.name.rstrip("0123456789"))
    assert kinds == {"cube", "plummer"}


@pytest.mark.parametrize("precision,tol", [(rp.RPY_FP64, 1e-12), (rp.RPY_FP32, 1e-6)])
def test_full_matvec_equals_near_plus_far_parts(precision, tol):
    """The full matvec sums each leaf's U list and its direct substitutes of small W / X
    interactions in one near-field pass; the part calls keep them apart (NEAR: U lists and
    self term; FAR: everything else, direct substitutes included).  Both splits add up to the
    same velocity, up to the rounding that regrouping the sums allows."""
    import torch
    sysm = synth.sphere_plus_cube(30000, 51, 1e-4)
    t = rp.rpy_forest_build(cuda_tensor(sysm.pos), [0, sysm.n], [sysm.a], 6, precision=precision, leaf_cap=40,
                            direct_w=200, direct_x=60)
    st = rp.rpy_tree_stats(t)
    assert st["n_dlist"] > 0 and st["d_pairs"] > 0
    F = cuda_tensor(sysm.f)
    out = {}
    for name, part in (("all", rp.RPY_PART_ALL), ("near", rp.RPY_PART_NEAR), ("far", rp.RPY_PART_FAR)):
        U = torch.empty_like(F)
        rp.rpy_matvec_parts(t, F, sysm.s, U, part)
        rp.rpy_tree_sync(t)
        out[name] = U.cpu().numpy()
    assert oracle.rel_l2(out["near"] + out["far"], out["all"]) < tol
    assert oracle.rel_l2(out["far"], out["all"]) > 1e-3   # the far part is not negligible


# ---------------------------------------------------------------- polynomial (Cartesian) far field

def test_cartesian_far_field_meets_3digits_and_converges_in_order():
    """RPY_FLAG_CARTESIAN (the polynomial expansions Sec. 5 proposes for low accuracy):
    at its default total degree the full velocity meets rel-L2 <= 1e-3 against the oracle
    in FP64 and FP32; the error falls geometrically with the degree (each +2 at least 2x);
    FP32 and FP64 differ only by rounding."""
    sysm = synth.config1()
    ref = oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s)
    errs = {}
    for P in (4, 6, 8, 10):
        u, t = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3, leaf_cap=40, order_p=P, flags=rp.RPY_FLAG_CARTESIAN)
        errs[P] = oracle.rel_l2(u, ref)
        assert rp.rpy_tree_stats(t)["n_vpairs"] > 0
    assert all(errs[P + 2] < 0.5 * errs[P] for P in (4, 6, 8)), errs
    u64, t64 = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3, leaf_cap=40, flags=rp.RPY_FLAG_CARTESIAN)
    u32, t32 = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3, leaf_cap=40, flags=rp.RPY_FLAG_CARTESIAN,
                      precision=rp.RPY_FP32)
    assert rp.rpy_tree_stats(t64)["order_p"] == 8
    assert oracle.rel_l2(u64, ref) < 1e-3 and oracle.rel_l2(u32, ref) < 1e-3
    assert oracle.rel_l2(u32, u64) < 1e-6


def test_cartesian_adaptive_sphere_and_dipole_regime():
    """The polynomial far field on an adaptive sphere-plus-cube tree (W and X lists summed
    directly) on sampled targets, and with a comparable to the box size (the a^2/r^2 term
    of Eq. (2.8) large), both at 3 digits against the oracle."""
    sysm = synth.sphere_plus_cube(200000, 71, 1e-4)
    tg = synth.sample_targets(sysm.n, 600)
    e, e_far, t = _check(sysm.pos, sysm.f, sysm.a, sysm.s, 3, 1e-3, targets=tg, precision=rp.RPY_FP32,
                         flags=rp.RPY_FLAG_CARTESIAN)
    st = rp.rpy_tree_stats(t)
    assert st["n_wlist"] == 0 and st["n_dlist"] > 0 and st["depth"] >= 5
    rng = np.random.default_rng(6)
    pos = rng.random((512, 3))
    f = rng.standard_normal((512, 3))
    a = 0.02
    _check(pos, f, a, 6 * math.pi * a, 3, 1e-3, leaf_cap=8, order_p=10, flags=rp.RPY_FLAG_CARTESIAN)


def test_cartesian_refusals():
    import torch
    sysm = synth.config1()
    P = cuda_tensor(sysm.pos)
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 6, flags=rp.RPY_FLAG_CARTESIAN)
    assert e.value.status == -2
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 3, order_p=11, flags=rp.RPY_FLAG_CARTESIAN)
    assert e.value.status == -1
    t = rp.rpy_forest_build(P, [0, sysm.n], [sysm.a], 3, leaf_cap=40, flags=rp.RPY_FLAG_CARTESIAN)
    q = torch.zeros((sysm.n, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((sysm.n, 52), dtype=torch.float64, device="cuda")
    with pytest.raises(rp.RpyError) as e:
        rp.rpy_laplace_far(t, q, out)
    assert e.value.status == -7
    t.close()


def test_bounded_device_wait_times_out_and_context_stays_usable():
    """The pipelined kernels' mbarrier waits are bounded: a wait that nothing completes gives up
    after its limit and reports RPY_ERR_TIMEOUT through the status word; the next matvec runs."""
    import time
    t0 = time.perf_counter()
    assert rp.rpy_debug_wait_timeout(50.0) == -5
    assert time.perf_counter() - t0 < 5.0
    sysm = synth.config1()
    u, t = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3, leaf_cap=40)
    assert oracle.rel_l2(u, oracle.rpy_direct(sysm.pos, sysm.f, sysm.a, sysm.s)) < 1e-3


def test_tree_work_counts_match_the_tree():
    """rpy_tree_work's per-stage numerators follow the tree: the near field counts 38 FLOP
    (FP64) or 33 (FP32) per near-list pair and 72 / 60 B per bead; every far-field stage of an
    FMM tree has work; the Cartesian form counts its multipole-to-local step under X2L from the
    V-list pairs, with nothing under M2X, X2X and P2L."""
    sysm = synth.sphere_plus_cube(50000, 81, 1e-4)
    for prec, per_pair, per_bead in ((rp.RPY_FP64, 38.0, 72.0), (rp.RPY_FP32, 33.0, 60.0)):
        u, t = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 6, leaf_cap=40, precision=prec)
        st = rp.rpy_tree_stats(t)
        w = rp.rpy_tree_work(t)
        assert w["p2p"][0] == per_pair * (st["u_pairs"] + st["d_pairs"])
        assert w["p2p"][1] == per_bead * sysm.n
        for k in ("p2m", "m2m", "m2x", "x2x", "x2l", "l2l", "eval"):
            assert w[k][0] > 0 and w[k][1] > 0, k
    u, t = matvec(sysm.pos, sysm.f, sysm.a, sysm.s, 3, leaf_cap=40, flags=rp.RPY_FLAG_CARTESIAN)
    st = rp.rpy_tree_stats(t)
    w = rp.rpy_tree_work(t)
    P = st["order_p"]
    terms = sum(math.comb(P - d + 3, 3) * (d + 1) * (d + 2) // 2 for d in range(P + 1))   # |a| + |b| <= P
    assert terms == math.comb(P + 6, 6)
    assert w["x2l"][0] == st["n_vpairs"] * terms * 4 * 2
    assert w["m2x"] == (0.0, 0.0) and w["x2x"] == (0.0, 0.0) and w["p2l"] == (0.0, 0.0)
