"""Pins of the block-sparse Theta_c application (oracle.blocksparse; CPU only).

Checked against the dense application of ``oracle.boundary`` (a different code
path: layered einsums over whole tensors) on charge-conserving inputs from the
U(1) x U(1) generators: equality for every sector, tasks with non-overlapping
outputs that cover the support of the result, fewer flops than the dense form,
and a planted bookkeeping mistake (a task that overwrites its block products instead of
summing them) that breaks the equality.
"""
import numpy as np
import pytest

from oracle import blocksparse as BS
from oracle import boundary as B
from oracle import symmetric as S
from synth import lattice as L
from synth import u1


def _setup(seed=3, Lx=3, Ly=3, D=2, c=1, boundary="random"):
    """Inputs of Theta_c at site c of row 1. boundary="random": a random charge-conserving boundary
    tensor with the charges and shape of the exact row-0 one (whose nonzero slices all have
    Q_U = 0 on this lattice, so it would leave the U-leg bookkeeping unexercised); "row0": that
    exact boundary tensor."""
    peps, ch = u1.u1_peps(Lx, Ly, D, seed)
    qpeps = [[u1.peps_leg_charges(ch, Lx, Ly, r, cc) for cc in range(Ly)] for r in range(Lx)]
    ham = L.hubbard_hamiltonian(Lx, Ly, seed)
    W, qW = L.fsm_pepo(ham), u1.hubbard_pepo_charges(ham)
    T, _ = B.first_row_boundary(peps[0], W[0])
    QL0, QU0, QR0, QD0 = S.site_bundles(qpeps[0][c], qW[0][c])
    qsite = S.site_bundles(qpeps[1][c], qW[1][c])
    Tc = T[c]
    g = np.random.default_rng(seed)
    if boundary == "random":
        rule = np.all(QL0[:, None, None, :] == QD0[None, :, None, :] + QR0[None, None, :, :], axis=-1)
        Tc = g.standard_normal(Tc.shape) * rule
    # left environment: charges a drawn from the reachable q_t + Q_L, entries off the rule zero
    reach = sorted({tuple(x) for x in (QL0[:, None, :] + qsite[0][None, :, :]).reshape(-1, 2).tolist()})
    qa = np.array([reach[i] for i in g.integers(0, len(reach), 14)], dtype=np.int64)
    EL = g.standard_normal((len(qa), Tc.shape[0], len(qsite[0])))
    ok = np.all(qa[:, None, None, :] == QL0[None, :, None, :] + qsite[0][None, None, :, :], axis=-1)
    EL = EL * ok
    return EL, qa, Tc, QL0, QD0, QR0, peps[1][c], W[1][c], qsite, g


def _sector_vectors(g, qtp, QR, q, k=3):
    X = g.standard_normal((len(qtp), len(QR), k))
    ok = np.all(qtp[:, None, :] + QR[None, :, :] == np.asarray(q), axis=-1)
    return X * ok[:, :, None]


def test_inputs_obey_the_charge_rules():
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, _ = _setup(boundary="row0")
    assert np.array_equal(qsite[1], qU)                       # the boundary's bundle meets the row's up legs
    rule = np.all(qt[:, None, None, :] == qU[None, :, None, :] + qtp[None, None, :, :], axis=-1)
    assert np.all(rule[Tc != 0]) and np.any(Tc != 0)


@pytest.mark.parametrize("seed,boundary", [(3, "random"), (5, "random"), (3, "row0")])
def test_block_application_equals_dense_for_every_sector(seed, boundary):
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, g = _setup(seed, boundary=boundary)
    QR = qsite[2]
    sectors = sorted({tuple(x) for x in (qtp[:, None, :] + QR[None, :, :]).reshape(-1, 2).tolist()})
    assert len(sectors) > 2
    for q in sectors:
        X = _sector_vectors(g, qtp, QR, q)
        yd = B.theta(EL, Tc, A, W, X)
        yb, tasks = BS.theta_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
        assert np.allclose(yb, yd, atol=1e-12 * max(1.0, np.abs(yd).max())), q
        # the dense result lives in the sector's rows only
        rows_ok = np.all(qa[:, None, :] - qsite[3][None, :, :] == np.asarray(q), axis=-1)
        assert np.all(yd[~rows_ok] == 0)


def test_tasks_are_disjoint_and_cover_the_result():
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, g = _setup(5)
    QR, QD = qsite[2], qsite[3]
    q = tuple((qtp[0] + QR[0]).tolist())
    X = _sector_vectors(g, qtp, QR, q)
    yd = B.theta(EL, Tc, A, W, X)
    _, tasks = BS.theta_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
    for step in (1, 2, 3):
        keys = [t.out for t in tasks if t.step == step]
        assert keys and len(keys) == len(set(keys)), step
    covered = np.zeros(yd.shape[:2], dtype=bool)
    ga, gd = BS.charge_groups(qa), BS.charge_groups(QD)
    for t in tasks:
        if t.step == 3:
            ca, cd = t.out
            covered[np.ix_(ga[ca], gd[cd])] = True
    assert np.all(covered[np.any(yd != 0, axis=2)])
    assert sum(t.flops for t in tasks) < BS.dense_flops(EL, Tc, A, W, X)


def test_planted_overwrite_instead_of_accumulate_is_caught(monkeypatch):
    """A task that keeps only its last block product (the sandwich and environment steps sum
    several) no longer equals the dense application."""
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, g = _setup(3)
    QR = qsite[2]
    q = (0, -1)
    X = _sector_vectors(g, qtp, QR, q)
    yd = B.theta(EL, Tc, A, W, X)
    _, tasks = BS.theta_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
    assert any(t.terms > 1 for t in tasks if t.step == 2) and any(t.terms > 1 for t in tasks if t.step == 3)
    monkeypatch.setattr(BS, "_accumulate", lambda acc, p: p)
    yb, _ = BS.theta_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
    assert not np.allclose(yb, yd, atol=1e-12 * np.abs(yd).max())


@pytest.mark.parametrize("seed", [3, 5])
def test_transpose_block_application_equals_dense_for_every_sector(seed):
    """Theta_c^T by charge blocks against the dense transpose application, every sector; its
    tasks are disjoint per step, and <Y, Theta X> = <Theta^T Y, X> holds on the block results."""
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, g = _setup(seed)
    QR, QD = qsite[2], qsite[3]
    sectors = sorted({tuple(x) for x in (qa[:, None, :] - QD[None, :, :]).reshape(-1, 2).tolist()})
    assert len(sectors) > 2
    for q in sectors:
        Y = g.standard_normal((len(qa), len(QD), 3)) * np.all(qa[:, None, :] - QD[None, :, :] == np.asarray(q),
                                                              axis=-1)[:, :, None]
        zd = B.theta_t(EL, Tc, A, W, Y)
        zb, tasks = BS.theta_t_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, Y, q)
        assert np.allclose(zb, zd, atol=1e-12 * max(1.0, np.abs(zd).max())), q
        for step in (1, 2, 3):
            keys = [t.out for t in tasks if t.step == step]
            assert len(keys) == len(set(keys)), (q, step)
        X = _sector_vectors(g, qtp, QR, q)
        yb, _ = BS.theta_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
        lhs, rhs = float(np.sum(Y * yb)), float(np.sum(zb * X))
        assert abs(lhs - rhs) <= 1e-10 * (1.0 + abs(lhs)), q


def _right_env(g, qtp, QR, n=12):
    """A random right environment ER[a, t', R] with q_a = q_t' + Q_R."""
    reach = sorted({tuple(x) for x in (qtp[:, None, :] + QR[None, :, :]).reshape(-1, 2).tolist()})
    qa = np.array([reach[i] for i in g.integers(0, len(reach), n)], dtype=np.int64)
    ER = g.standard_normal((n, len(qtp), len(QR)))
    ok = np.all(qa[:, None, None, :] == qtp[None, :, None, :] + QR[None, None, :, :], axis=-1)
    return ER * ok, qa


@pytest.mark.parametrize("seed", [3, 5])
def test_right_environment_maps_by_blocks_equal_dense(seed):
    """ThetaR_c and its transpose by charge blocks against the dense maps, every sector, with
    disjoint tasks per step and the adjoint identity <Z, ThetaR X> = <ThetaR^T Z, X>."""
    _, _, Tc, qt, qU, qtp, A, W, qsite, g = _setup(seed)
    QL, _, QR, QD = qsite
    ER, qa = _right_env(g, qtp, QR)
    sectors = sorted({tuple(x) for x in (QD[:, None, :] + qa[None, :, :]).reshape(-1, 2).tolist()})
    assert len(sectors) > 2
    for q in sectors:
        X = g.standard_normal((len(QD), len(qa), 2)) * np.all(QD[:, None, :] + qa[None, :, :] == np.asarray(q),
                                                              axis=-1)[:, :, None]
        zd = B.theta_r(ER, Tc, A, W, X)
        zb, tasks = BS.theta_r_blocks(ER, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
        assert np.allclose(zb, zd, atol=1e-12 * max(1.0, np.abs(zd).max())), q
        Zin = g.standard_normal((len(qt), len(QL), 2)) * np.all(qt[:, None, :] + QL[None, :, :] == np.asarray(q),
                                                                axis=-1)[:, :, None]
        xd = B.theta_r_t(ER, Tc, A, W, Zin)
        xb, tasks_t = BS.theta_r_t_blocks(ER, qa, Tc, qt, qU, qtp, A, W, qsite, Zin, q)
        assert np.allclose(xb, xd, atol=1e-12 * max(1.0, np.abs(xd).max())), q
        for tl in (tasks, tasks_t):
            for step in (1, 2, 3):
                keys = [t.out for t in tl if t.step == step]
                assert len(keys) == len(set(keys)), (q, step)
        lhs, rhs = float(np.sum(Zin * zb)), float(np.sum(xb * X))
        assert abs(lhs - rhs) <= 1e-10 * (1.0 + abs(lhs)), q
