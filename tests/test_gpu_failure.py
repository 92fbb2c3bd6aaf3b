"""Failure paths of the CUDA library, through the C-ABI, with no GPU fault.

- Non-finite problem data (NaN in A or b) is reported as RAC_ERR_NUMERIC
  before any sweep runs, for the single-problem handle in both gradient forms
  and for one instance of a batch, whose other instances still converge.
- A bounded in-kernel wait that runs out is reported as RAC_ERR_TIMEOUT: the
  host-set option debug_exit_cta makes one CTA of the residual-form block
  chain leave before it ever arrives at a grid barrier, so every other CTA's
  wait ends at its limit (1 s) and the kernel returns.  The device stays
  usable: the next handle on it matches the oracle sweep for sweep.
"""
import time

import numpy as np
import pytest

import synth
from oracle import rac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01995_gb300 import _lib  # noqa: E402
from paper_1907_01995_gb300 import api  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


@pytest.mark.parametrize("where", ["A", "b"])
@pytest.mark.parametrize("form,storage", [("gram", "fp64"), ("gram", "bf16"),
                                          ("residual", "fp64"), ("residual", "fp32")])
def test_nonfinite_data_is_reported(where, form, storage):
    inst = synth.small_instance(6, 57, 43, 5)
    A, b = inst.A.copy(order="F"), inst.b.copy()
    if where == "A":
        A[11, 7] = np.nan
    else:
        b[3] = np.inf
    with api.Handle(A, b, phi="l1l2", lambda1=inst.lam1, num_blocks=5, tol=1e-8,
                    max_sweeps=50, form=form, storage=storage) as h:
        with pytest.raises(_lib.RacError) as ei:
            h.solve()
    assert ei.value.status == _lib.RAC_ERR_NUMERIC


def test_batch_nonfinite_instance_is_isolated():
    insts = [synth.small_instance(30 + i, 60 + 7 * i, 30 + 5 * i, 3 + i) for i in range(3)]
    probs = [dict(A=s.A.copy(order="F"), b=s.b, phi="l1l2", lambda1=s.lam1) for s in insts]
    probs[1]["A"][4, 9] = np.nan
    zs, infos = api.batch(probs, num_blocks=-8, beta=1.0, tol=1e-9, max_sweeps=5000,
                          refresh_every=10, storage="fp64",
                          allow=(_lib.RAC_OK, _lib.RAC_ERR_NUMERIC))
    assert infos[1]["status"] == _lib.RAC_ERR_NUMERIC
    assert infos[1]["sweeps"] == 0
    for i in (0, 2):
        assert infos[i]["status"] == 0, infos[i]
        ref = O.cd_enet(insts[i].A, insts[i].b, insts[i].lam1, 0.0)
        assert rel(zs[i], ref) <= 1e-6


def test_barrier_timeout_is_reported_and_device_stays_usable():
    inst = synth.small_instance(3, 57, 43, 5)
    kw = dict(phi="l1l2", lambda1=inst.lam1, num_blocks=5, beta=1.0, gamma=1.0,
              storage="fp64", form="residual", grid=4, refresh_every=5, seed=11)
    t0 = time.perf_counter()
    with api.Handle(inst.A, inst.b, tol=1e-8, max_sweeps=20, debug_exit_cta=3, **kw) as h:
        with pytest.raises(_lib.RacError) as ei:
            h.solve()
    elapsed = time.perf_counter() - t0
    assert ei.value.status == _lib.RAC_ERR_TIMEOUT
    # one barrier wait ran to its 1 s limit; the later launches of the period
    # saw the recorded status and returned at once
    assert elapsed < 20.0, elapsed
    # the context is intact: a fresh handle follows the oracle exactly
    P = O.problem_from_instance(inst)
    ost = O.initial_state(P)
    for _ in range(10):
        O.sweep(P, ost, 5, 11, 1.0, 1.0)
    with api.Handle(inst.A, inst.b, tol=0.0, max_sweeps=10, **kw) as h:
        _, info = h.solve()
        st = h.state()
    # tol = 0: the call runs its 10 sweeps and ends at the sweep cap
    assert info["sweeps"] == 10 and info["status"] == _lib.RAC_ERR_NOT_CONVERGED
    assert rel(st["z"], ost.z) <= 1e-10
