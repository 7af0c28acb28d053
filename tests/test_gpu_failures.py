"""Failure paths of the C ABI, with the failure made on the host (no GPU fault).

* An allocator that returns NULL: the call that needed the memory returns
  FPEPS_ERR_OOM, the env can still be destroyed, and a fresh env on the same
  context computes the right value.
* Non-finite input data (a NaN in a PEPS site, an Inf in a PEPO site): the
  sweep returns FPEPS_ERR_NUMERIC (detected by the finite checks of the
  normalisation and of the QR's Gram matrix), and the context stays usable.
"""
import math

import numpy as np
import pytest

from oracle import network as N
from synth import lattice as L

pytestmark = pytest.mark.gpu

OOM, NUMERIC = 3, 5


@pytest.fixture(scope="module")
def fp():
    import torch
    from paper_2511_01039_gb300 import fpeps
    torch.cuda.set_device(0)
    fpeps.lib()
    return fpeps


def _small():
    peps = L.random_peps(3, 3, 2, 4, seed=0)
    pepo = L.fsm_pepo(L.random_hamiltonian(3, 3, 4, 2, seed=1))
    return peps, pepo


def _check_fresh_env(fp, peps, pepo):
    num, den = N.brute_force_expectation(peps, pepo)
    env = fp.Env(peps, pepo, D=2, p=4, w=4, chi=256, prec="f64", seed=3)
    val, _, _ = env.expect(fp.params(10, 0, 0, 1, 1))
    env.close()
    assert abs(val / (num / den) - 1) < 1e-10


class _FailingAllocator:
    """Torch-backed allocator that returns NULL once `budget` allocations were made."""

    def __init__(self, fp, device, budget):
        self.inner = fp.TorchAllocator(device)
        self.budget = budget
        self.calls = 0
        self.failed = 0
        self._a = fp.ALLOC_FN(self._alloc)
        self._f = fp.FREE_FN(self._free)
        self.struct = fp.fpeps_allocator(None, self._a, self._f)

    def _alloc(self, ctx, nbytes, stream):
        self.calls += 1
        if self.budget is not None and self.calls > self.budget:
            self.failed += 1
            return None
        return self.inner._alloc(ctx, nbytes, stream)

    def _free(self, ctx, ptr, stream):
        self.inner._free(ctx, ptr, stream)


def _create(fp, peps, pepo, allocator, prec="f64"):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    pk = torch.cat([torch.as_tensor(t).reshape(-1) for row in peps for t in row]).to(dev)
    wk = torch.cat([torch.as_tensor(t).reshape(-1) for row in pepo for t in row]).to(dev)
    cfg = fp.fpeps_config(len(peps), len(peps[0]), 2, 4, 4, 256, fp.PRECISIONS[prec], 3, 0, 1)
    torch.cuda.synchronize()
    return fp.fpeps_env_create(cfg, pk, wk, 0, torch.cuda.current_stream().cuda_stream, allocator)


def test_allocator_null_at_create_is_err_oom(fp):
    import torch
    peps, pepo = _small()
    al = _FailingAllocator(fp, torch.device("cuda", 0), budget=2)
    with pytest.raises(fp.FpepsError) as ei:
        _create(fp, peps, pepo, al)
    assert ei.value.status == OOM and al.failed >= 1
    _check_fresh_env(fp, peps, pepo)


def test_allocator_null_during_sweep_is_err_oom(fp):
    import torch
    peps, pepo = _small()
    al = _FailingAllocator(fp, torch.device("cuda", 0), budget=None)
    h = _create(fp, peps, pepo, al)
    al.budget = al.calls + 3          # a few more blocks, then NULL in the middle of the sweep
    with pytest.raises(fp.FpepsError) as ei:
        fp.fpeps_expect(h, fp.params(10, 0, 0, 1, 1))
    assert ei.value.status == OOM and al.failed >= 1
    assert "NULL" in fp.fpeps_last_error(h) or "allocator" in fp.fpeps_last_error(h)
    fp.fpeps_env_destroy(h)
    _check_fresh_env(fp, peps, pepo)


@pytest.mark.parametrize("where", ["peps_row0", "peps_interior", "pepo_interior"])
@pytest.mark.parametrize("prec", ["f64", "tf32x3"])
def test_non_finite_input_is_err_numeric(fp, where, prec):
    peps, pepo = _small()
    peps = [[a.copy() for a in row] for row in peps]
    pepo = [[w.copy() for w in row] for row in pepo]
    if where == "peps_row0":
        peps[0][1].flat[3] = math.nan
    elif where == "peps_interior":
        peps[1][1].flat[5] = math.nan
    else:
        w = pepo[1][1]
        idx = np.argwhere(w != 0)[0]      # a structurally nonzero entry, so the channel is used
        w[tuple(idx)] = math.inf
    env = fp.Env(peps, pepo, D=2, p=4, w=4, chi=256, prec=prec, seed=3)
    with pytest.raises(fp.FpepsError) as ei:
        env.expect(fp.params(10, 0, 0, 1, 1))
    assert ei.value.status == NUMERIC
    env.close()
    _check_fresh_env(fp, *_small())
