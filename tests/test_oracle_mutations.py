"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each test patches one plausible error into the oracle (a transposed operand, a
dropped term, a wrong sign or index) and checks that the brute-force,
closed-form or exactness pin no longer holds. Nothing here touches a GPU.
"""
import math

import numpy as np
import pytest

from oracle import boundary as B
from oracle import network as N
from synth import lattice as L


def _boundary_value(peps, pepo, chi=256):
    s, lv = B.contract(peps, pepo, chi, B.RsvdParams(exact_svd=True, n_fit=1, power_iters=0), seed=3, layer=1)
    return s * math.exp(lv)


@pytest.fixture
def small():
    peps = L.random_peps(3, 3, 2, 4, seed=0)
    pepo = L.fsm_pepo(L.random_hamiltonian(3, 3, 4, 2, seed=1))
    num, _ = N.brute_force_expectation(peps, pepo)
    return peps, pepo, num


def test_unpatched_reference_holds(small):
    peps, pepo, num = small
    assert _boundary_value(peps, pepo) == pytest.approx(num, rel=1e-10)


def test_pepo_physical_leg_swap_is_a_symmetry_not_a_pin_gap():
    """p <-> p' exchanged in every PEPO block gives O^T, and <psi|O^T|psi> = <psi|O|psi> for real psi:
    this reading of the paper cannot change any value (documented reading, not a mistake)."""
    peps = L.random_peps(3, 3, 2, 4, seed=0)
    ham = L.hubbard_hamiltonian(3, 3, seed=2, K=4)     # c^dag / c blocks are not symmetric
    pepo = L.fsm_pepo(ham)
    swapped = [[np.swapaxes(w, 4, 5).copy() for w in row] for row in pepo]
    a, _ = N.brute_force_expectation(peps, pepo)
    b, _ = N.brute_force_expectation(peps, swapped)
    assert a == pytest.approx(b, rel=1e-12)


def test_wrong_bra_leg_is_caught(small, monkeypatch):
    """The bra with its left and right legs exchanged (a transposed operand) breaks pin (a)."""
    peps, pepo, num = small
    orig = N.sandwich_apply

    def wrong(G, A, W, ins, outs):
        if A.shape[0] == A.shape[2]:
            A = np.ascontiguousarray(np.swapaxes(A, 0, 2))
        return orig(G, A, W, ins, outs)

    monkeypatch.setattr(B, "sandwich_apply", wrong)
    assert _boundary_value(peps, pepo) != pytest.approx(num, rel=1e-6)


def test_dropped_hopping_term_in_fsm_is_caught():
    ham = L.random_hamiltonian(3, 3, 4, 2, seed=4)
    peps = L.random_peps(3, 3, 2, 4, seed=4)
    good = L.fsm_pepo(ham)
    bad = [[w.copy() for w in row] for row in good]
    # remove the vertical completion X^0 -> D at site (1,1): a dropped term
    W = bad[1][1]
    N_, Dn, I_ = 0, 1, 0
    W[N_, 1 + 0, Dn, I_] = 0.0
    psi = N.psi_vector(peps)
    ref = psi @ N.apply_terms(psi, ham)
    assert N.brute_force_expectation(peps, good)[0] == pytest.approx(ref, rel=1e-10)
    assert N.brute_force_expectation(peps, bad)[0] != pytest.approx(ref, rel=1e-6)


def test_wrong_sign_in_cbe_projection_is_caught():
    """Fig. 5 subtraction with a + instead of a -: the explicit-projector identity fails."""
    g = np.random.default_rng(1)
    m, n, a = 20, 16, 4
    th2 = g.standard_normal((m, n))
    V = np.linalg.qr(g.standard_normal((n, a)))[0].T
    om = g.standard_normal((n, 5))
    explicit = th2 @ (np.eye(n) - V.T @ V) @ om
    assert np.allclose(th2 @ om - th2 @ (V.T @ (V @ om)), explicit)
    assert not np.allclose(th2 @ om + th2 @ (V.T @ (V @ om)), explicit)


def test_off_by_one_sketch_counter_is_caught():
    """Shifting the Philox counter by one breaks the numpy known-answer test."""
    from oracle.philox import philox4x64_10
    key = np.array([3, 5], dtype=np.uint64)
    bg = np.random.Philox(key=key, counter=np.array([0, 0, 0, 0], dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(4)]
    good = [int(x[0]) for x in philox4x64_10(tuple(np.array([v], dtype=np.uint64) for v in (1, 0, 0, 0)), key)]
    bad = [int(x[0]) for x in philox4x64_10(tuple(np.array([v], dtype=np.uint64) for v in (0, 0, 0, 0)), key)]
    assert good == raw and bad != raw


def test_arbitrary_qr_completion_is_caught(monkeypatch):
    """Householder's arbitrary completion directions for a rank-deficient Y (the
    reading the oracle rejects) fail the zero-column pin; an unordered basis of
    the same span (an SVD) fails the LAPACK-order pin."""
    import tests.test_oracle_pins as P

    def householder(Y):
        Q, R = np.linalg.qr(Y)
        return Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]

    def svd_basis(Y):
        return np.linalg.svd(Y, full_matrices=False)[0]

    monkeypatch.setattr(B, "orth", householder)
    with pytest.raises(AssertionError):
        P.test_orth_dependent_columns_become_zero()
    monkeypatch.setattr(B, "orth", svd_basis)
    with pytest.raises(AssertionError):
        P.test_orth_full_rank_is_lapack_thin_qr()
