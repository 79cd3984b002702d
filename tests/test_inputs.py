"""The seeded input recipe holds what it promises (CPU): compositions, electron and AO counts of
the fixed workloads, the covalent-walk geometry rules, the basis rule, orbitals orthonormal in
the AO overlap metric, walkers drawn round-robin around the nuclei, and the ranges of the
ragged batch."""
import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S


def _pair_distances(R):
    d = np.linalg.norm(R[:, None, :] - R[None, :, :], axis=-1)
    return d[np.triu_indices(len(R), 1)]


@pytest.mark.parametrize("cfg,Ne,M,K", [(0, 10, 24, 3), (1, 26, 72, 9), (4, 94, 222, 21)])
def test_fixed_workloads_have_their_sizes(cfg, Ne, M, K):
    sx = S.make_system(cfg)
    assert (sx.Ne, sx.M, sx.K) == (Ne, M, K)
    assert sx.n_up == sx.n_dn == Ne // 2
    assert int(sx.Z.sum()) == Ne  # neutral, all-electron


def test_water_geometry_is_the_jittered_reference():
    Z, R = S.water_geometry(np.random.default_rng(0))
    assert list(Z) == [8, 1, 1]
    ref = np.array([[0.0, 0.0, 0.0], [1.81, 0.0, 0.0],
                    [1.81 * np.cos(np.radians(104.5)), 1.81 * np.sin(np.radians(104.5)), 0.0]])
    assert np.abs(R - ref).max() <= 0.05


@pytest.mark.parametrize("cfg", [1, 4])
def test_covalent_walk_rules(cfg):
    sx = S.make_system(cfg)
    R, Z = sx.R, np.asarray(sx.Z)
    assert _pair_distances(R).min() >= 1.7 - 1e-12
    heavy = np.flatnonzero(Z > 1)
    # every atom but the first sits at a bond length from some heavy atom
    for i in range(1, len(Z)):
        d = np.linalg.norm(R[heavy] - R[i], axis=1)
        d = d[heavy != i]
        assert np.any((d >= 1.9 - 1e-9) & (d <= 2.9 + 1e-9)), i


def test_basis_rule_shells_and_exponent_ranges():
    Z = np.array([8, 6, 1])
    c, l, npr, ex, co = S.basis_rule(Z, np.random.default_rng(5))
    assert list(l) == [0, 0, 0, 1, 1, 2] * 2 + [0, 0, 1]
    assert list(c) == [0] * 6 + [1] * 6 + [2] * 3
    assert np.all(npr == S.MAXPRIM)
    assert np.all(np.diff(ex, axis=1) <= 0)  # sorted descending per shell
    assert ex.min() >= 0.1
    assert ex[:3].max() <= 5000.0 and ex[3:].max() <= 30.0  # only O s shells reach past 30
    assert co.min() >= 0.2 and co.max() <= 1.0


@pytest.mark.parametrize("cfg", [0, 1])
def test_orbitals_are_orthonormal_in_the_overlap_metric(cfg):
    sx = S.make_system(cfg)
    Sm = S.overlap_matrix(sx)
    assert np.allclose(Sm, Sm.T, atol=1e-12)
    assert np.allclose(np.diag(Sm), 1.0, atol=1e-10)  # normalised AOs
    for C in (sx.C_up, sx.C_dn):
        assert np.abs(C.T @ Sm @ C - np.eye(C.shape[1])).max() < 1e-9
    assert not np.allclose(sx.C_up, sx.C_dn)  # independent draws per spin


def test_walkers_are_drawn_round_robin_around_the_nuclei():
    sx = S.make_system(1)
    pos = S.initial_walkers(sx, 4096, seed=3)
    assert pos.shape == (4096, sx.Ne, 3)
    for e in range(sx.Ne):
        d = pos[:, e, :] - sx.R[e % sx.K]
        assert abs(d.mean()) < 0.05 and abs(d.std() - 1.0) < 0.05
    np.testing.assert_array_equal(pos, S.initial_walkers(sx, 4096, seed=3))


def test_ragged_batch_plan_ranges():
    plan = S.ragged_batch_plan()
    assert len(plan) == 64
    for Z, W in plan:
        ne = sum(Z)
        assert 3 <= len(Z) <= 21 and Z[0] in (6, 8) and set(Z) <= {1, 6, 8}
        assert ne % 2 == 0 and 10 <= ne <= 94
        assert 512 <= W <= 4096 and W % 128 == 0
