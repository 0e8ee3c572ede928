"""Failure detection without a GPU fault: host-side fault injection through
CHI0_FAULT and the bounded device waits, whose expiry is reported as a status
(the wait self-test uses a barrier that nothing releases; no trap, no hang)."""
import ctypes as C
import os

import numpy as np
import pytest

import paper_1601_06767_gb300 as pkg
from paper_1601_06767_gb300 import _lib as L
from synth import make_problem


def _desc(prob, keep):
    d = L.Chi0PlanDesc()
    g = np.ascontiguousarray(prob.gvec[0].astype(np.int32))
    nG = np.array([g.shape[0]], np.int32)
    re = np.ascontiguousarray(prob.omega.real)
    im = np.ascontiguousarray(prob.omega.imag)
    keep += [g, nG, re, im]
    d.n1 = d.n2 = d.n3 = prob.n
    d.n_q = 1
    d.n_G = nG.ctypes.data_as(C.POINTER(C.c_int32))
    d.gvec = g.ctypes.data_as(C.POINTER(C.c_int32))
    d.n_freq = re.size
    d.freq_re = re.ctypes.data_as(C.POINTER(C.c_double))
    d.freq_im = im.ctypes.data_as(C.POINTER(C.c_double))
    d.delta = prob.delta
    return d


def test_injected_bad_shape_is_reported_before_any_device_work(monkeypatch):
    monkeypatch.setenv("CHI0_FAULT", "bad_shape")
    keep = []
    d = _desc(make_problem("c1"), keep)
    h = C.c_void_p()
    assert pkg.lib().chi0_plan_create(C.byref(h), C.byref(d)) == L.CHI0_ERR_INVALID
    assert b"injected" in pkg.lib().chi0_last_error(None)
    assert h.value is None


@pytest.mark.gpu
def test_injected_oom_frees_everything(monkeypatch):
    monkeypatch.setenv("CHI0_FAULT", "oom")
    keep = []
    d = _desc(make_problem("c1"), keep)
    h = C.c_void_p()
    assert pkg.lib().chi0_plan_create(C.byref(h), C.byref(d)) == L.CHI0_ERR_OOM
    assert h.value is None
    monkeypatch.delenv("CHI0_FAULT")
    assert pkg.lib().chi0_plan_create(C.byref(h), C.byref(d)) == L.CHI0_OK
    pkg.lib().chi0_plan_destroy(h)


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_plan_stays_usable():
    import torch
    from oracle import chi0_from_pairs, freq_factor, rel_fro
    prob = make_problem("c1", n_imag=1)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    with pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp16") as plan:
        assert pkg.lib().chi0_selftest_wait(plan._h, 5.0, stream) == L.CHI0_OK
        with pytest.raises(pkg.Chi0Error) as ei:
            plan.sync_status()
        assert ei.value.status == L.CHI0_ERR_TIMEOUT
        plan.sync_status()            # the status was cleared
        rng = np.random.default_rng(0)
        M = (rng.standard_normal((64, 350)) + 1j * rng.standard_normal((64, 350))) * 0.01
        Ev, Ec = prob.E_v[:4], prob.E_c[:16]
        dE = (Ev[:, None] - Ec[None, :]).reshape(-1)
        ref = chi0_from_pairs(M, freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta))
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        chi = plan.accumulate(0, d(M.astype(np.complex64)), 4, 16, d(Ev), d(Ec))
        plan.sync_status()
        assert max(rel_fro(chi[i].cpu().numpy(), ref[i]) for i in range(2)) < 1e-6
