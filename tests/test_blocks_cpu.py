"""The library's task table of the block-sparse Theta_c application (host code, no GPU)
against the oracle's block-sparse application (oracle.blocksparse), which builds its tasks
independently while it computes: same tasks in the same order, same numbers of block
products, same flops, for every sector of the charged test lattices."""
import numpy as np
import pytest

from oracle import blocksparse as BS
from test_oracle_blocksparse import _right_env, _sector_vectors, _setup


@pytest.fixture(scope="module")
def fp():
    from paper_2511_01039_gb300 import build
    build.build()
    from paper_2511_01039_gb300 import fpeps
    return fpeps


@pytest.mark.parametrize("seed", [3, 5])
def test_task_table_matches_the_oracle(fp, seed):
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, g = _setup(seed)
    QL, _, QR, QD = qsite
    sectors = sorted({tuple(x) for x in (qtp[:, None, :] + QR[None, :, :]).reshape(-1, 2).tolist()})
    k = 3
    for q in sectors:
        X = _sector_vectors(g, qtp, QR, q, k=k)
        _, ref = BS.theta_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, X, q)
        got = fp.fpeps_theta_block_tasks(qa, qt, qU, qtp, QL, QR, QD, q)
        assert len(got) == len(ref), q
        for (step, terms, out, fl), t in zip(got, ref):
            assert (step, terms, out) == (t.step, t.terms, tuple(t.out)), q
            assert fl * k == pytest.approx(t.flops, rel=1e-12)


def test_task_table_arguments(fp):
    import ctypes
    one = np.zeros((1, 2), dtype=np.int32)
    assert fp.fpeps_theta_block_tasks(one, one, one, one, one, one, one, (0, 0)) == [
        (1, 1, ((0, 0), (0, 0), (0, 0)), 2.0), (2, 1, ((0, 0), (0, 0), (0, 0)), 2.0), (3, 1, ((0, 0), (0, 0)), 2.0)]
    # a sector no column carries: no tasks
    assert fp.fpeps_theta_block_tasks(one, one, one, one, one, one, one, (1, 0)) == []
    n = ctypes.c_int32(1)
    p = one.ctypes.data
    # capacity 1 for three tasks, and an empty leg
    buf = np.zeros((1, 8), dtype=np.int32)
    fl = np.zeros(1)
    args = [p, 1] * 7
    assert fp.lib().fpeps_theta_block_tasks(0, *args, p, buf.ctypes.data, fl.ctypes.data, ctypes.byref(n)) == 1
    n = ctypes.c_int32(0)
    assert fp.lib().fpeps_theta_block_tasks(4, *args, p, None, None, ctypes.byref(n)) == 1   # unknown op
    args[1] = 0
    assert fp.lib().fpeps_theta_block_tasks(0, *args, p, None, None, ctypes.byref(n)) == 1


@pytest.mark.parametrize("seed", [3, 5])
def test_transpose_task_table_matches_the_oracle(fp, seed):
    EL, qa, Tc, qt, qU, qtp, A, W, qsite, g = _setup(seed)
    QL, _, QR, QD = qsite
    sectors = sorted({tuple(x) for x in (qa[:, None, :] - QD[None, :, :]).reshape(-1, 2).tolist()})
    k = 2
    for q in sectors:
        Y = g.standard_normal((len(qa), len(QD), k))
        _, ref = BS.theta_t_blocks(EL, qa, Tc, qt, qU, qtp, A, W, qsite, Y, q)
        got = fp.fpeps_theta_block_tasks(qa, qt, qU, qtp, QL, QR, QD, q, op=1)
        assert len(got) == len(ref), q
        for (step, terms, out, fl), t in zip(got, ref):
            assert (step, terms, out) == (t.step, t.terms, tuple(t.out)), q
            assert fl * k == pytest.approx(t.flops, rel=1e-12)


@pytest.mark.parametrize("seed", [3, 5])
def test_right_environment_task_tables_match_the_oracle(fp, seed):
    _, _, Tc, qt, qU, qtp, A, W, qsite, g = _setup(seed)
    QL, _, QR, QD = qsite
    ER, qa = _right_env(g, qtp, QR)
    sectors = sorted({tuple(x) for x in (QD[:, None, :] + qa[None, :, :]).reshape(-1, 2).tolist()})
    for q in sectors:
        X = g.standard_normal((len(QD), len(qa), 1))
        Z = g.standard_normal((len(qt), len(QL), 1))
        for op, fn, v in ((2, BS.theta_r_blocks, X), (3, BS.theta_r_t_blocks, Z)):
            _, ref = fn(ER, qa, Tc, qt, qU, qtp, A, W, qsite, v, q)
            got = fp.fpeps_theta_block_tasks(qa, qt, qU, qtp, QL, QR, QD, q, op=op)
            assert len(got) == len(ref), (op, q)
            for (step, terms, out, fl), t in zip(got, ref):
                assert (step, terms, out) == (t.step, t.terms, tuple(t.out)), (op, q)
                assert fl == pytest.approx(t.flops, rel=1e-12)
