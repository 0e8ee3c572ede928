"""The allocation-free FP64 accumulate (chi0_accumulate_fp64_noalloc) against
the plan-based chi0_accumulate of a CHI0_FP64 plan and against the FP64
oracle of Eq. 1.

That entry point is for callers that cannot allocate device memory when they
need chi0 (a framework that owns all device memory, a loop that must not call
cudaMalloc); its only scratch is a fixed array inside the library.  Two calls
in a row check that the shared array's leftover contents do not leak into the
next result.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from oracle import chi0_from_pairs, freq_factor
from synth import make_problem

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_matches_plan_accumulate_twice():
    import torch
    import paper_1601_06767_gb300 as pkg
    from paper_1601_06767_gb300 import _lib as L

    lib = pkg.lib()
    prob = make_problem("c1", n_G=[203], n_imag=40)      # 41 frequencies: several scratch chunks
    nG, nf = prob.gvec[0].shape[0], prob.omega.size
    rng = np.random.default_rng(7)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    re = np.ascontiguousarray(prob.omega.real)
    im = np.ascontiguousarray(prob.omega.imag)
    cases = [(9, 1500, True), (4, 333, False)]           # 13,500 and 1,332 pairs; 2^18/41 = 6393 per chunk
    for call, (nv, nc, weighted) in enumerate(cases):
        M = (rng.standard_normal((nv * nc, nG)) + 1j * rng.standard_normal((nv * nc, nG))) * 0.05
        Ev = prob.E_v[:nv] if nv <= prob.n_v else rng.uniform(-0.25, 0, nv)
        Ec = np.sort(rng.uniform(0.17, 2.2, nc))
        w = rng.uniform(0.5, 30.0, nc) if weighted else None
        d = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
        Md, Evd, Ecd, wd = d(M), d(Ev), d(Ec), d(w)
        with pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp64") as plan:
            ref = plan.accumulate(0, Md, nv, nc, Evd, Ecd, wd)
            plan.sync_status()
        got = torch.zeros_like(ref)
        st = lib.chi0_accumulate_fp64_noalloc(nG, C.c_void_p(Md.data_ptr()), nv, nc, C.c_void_p(Evd.data_ptr()),
                                              C.c_void_p(Ecd.data_ptr()),
                                              None if wd is None else C.c_void_p(wd.data_ptr()), nf,
                                              re.ctypes.data, im.ctypes.data, prob.delta,
                                              C.c_void_p(got.data_ptr()), stream)
        assert st == L.CHI0_OK, lib.chi0_last_error(None)
        torch.cuda.synchronize()
        got_h = got.cpu().numpy()
        err = max(_rel(got_h[i], ref[i].cpu().numpy()) for i in range(nf))
        assert err < TOL64, (call, err)
        # and against the FP64 oracle of Eq. 1 directly
        dE = (Ev[:, None] - Ec[None, :]).reshape(-1)
        wp = np.tile(w, nv) if weighted else np.ones_like(dE)
        oracle = chi0_from_pairs(M, freq_factor(dE, wp, prob.omega, prob.delta))
        err_o = max(_rel(got_h[i], oracle[i]) for i in range(nf))
        assert err_o < TOL64, (call, err_o)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import paper_1601_06767_gb300 as pkg
    from paper_1601_06767_gb300 import _lib as L
    lib = pkg.lib()
    f = np.zeros(65)
    st = lib.chi0_accumulate_fp64_noalloc(10, C.c_void_p(16), 1, 1, C.c_void_p(16), C.c_void_p(16), None, 65,
                                          f.ctypes.data, f.ctypes.data, 1e-3, C.c_void_p(16), None)
    assert st == L.CHI0_ERR_INVALID
    assert b"fixed limit" in lib.chi0_last_error(None)
