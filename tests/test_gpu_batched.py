"""Batched build (one persistent tensor-core launch over all q-points and
frequencies per conduction block, captured in a CUDA graph) against the FP64
oracle and against the single-q build.  q-points on a shifted 2x2x2 grid with
uneven sphere sizes."""
import numpy as np
import pytest

from _parity import check_chi
from oracle import chi0_from_pairs, freq_factor, pair_elements, rel_fro, wfn_to_grid
from synth import make_problem

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,nG,nv,nc,n_imag", [
    ("c1", [150 + 25 * j for j in range(8)], 3, 40, 3),     # 8 q-points, N_G 150..325
    ("c3", [2200, 2600], 2, 12, 1),                         # the batched workload's smallest / largest spheres
])
@pytest.mark.parametrize("precision", ["fp16", "bf16"])    # bf16: Hermitian mode (upper tiles, H1 + i H2)
def test_batched_matches_oracle_and_single_q(name, nG, nv, nc, n_imag, precision):
    import torch
    from paper_1601_06767_gb300 import Chi0Plan
    qf = [((i + 0.5) / 2, (j + 0.5) / 2, (l + 0.5) / 2) for i in range(2) for j in range(2) for l in range(2)]
    prob = make_problem(name, n_G=nG, q_frac=qf[:len(nG)], n_imag=n_imag)
    nq = prob.n_q
    cc = prob.coeff_c(np.arange(nc))
    uc = wfn_to_grid(cc, prob.gw, prob.n)
    Ev, Ec = prob.E_v[:nv], prob.E_c[:nc]
    dE = (Ev[:, None] - Ec[None, :]).reshape(-1)
    f = freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta)
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=precision, gw=prob.gw, max_pairs=64) as plan:
        psi_c = plan.wfn_to_grid(_dev(cc))
        psi_vs = [plan.wfn_to_grid(_dev(prob.coeff_v(q, np.arange(nv)))) for q in range(nq)]
        Evs = [_dev(Ev) for _ in range(nq)]
        chis = plan.build_batched(psi_vs, Evs, psi_c, _dev(Ec), use_graph=True)
        plan.sync_status()
        got = [c.cpu().numpy() for c in chis]
        # the graph again, on zeroed outputs
        for c in chis:
            c.zero_()
        plan.build_batched(psi_vs, Evs, psi_c, _dev(Ec), chis=chis, use_graph=True)
        plan.sync_status()
        again = [c.cpu().numpy() for c in chis]
        single = [plan.build(q, psi_vs[q], Evs[q], psi_c, _dev(Ec)).cpu().numpy() for q in range(nq)]
        plan.sync_status()
    for q in range(nq):
        uv = wfn_to_grid(prob.coeff_v(q, np.arange(nv)), prob.gw, prob.n)
        ref = chi0_from_pairs(pair_elements(uv, uc, prob.gvec[q], prob.n), f)
        check_chi(got[q], ref, TOL, label=f"batched {name} {precision} q{q}")
        assert np.array_equal(got[q], again[q])
        assert np.array_equal(got[q], single[q])


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    import torch
    from paper_1601_06767_gb300 import Chi0Plan
    monkeypatch.setenv("CHI0_TUNE_CACHE", str(tmp_path / "tune.txt"))
    prob = make_problem("c1", n_imag=2)
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp16", max_pairs=8192) as plan:
        t = plan.autotune(0, force=True)
        assert t["group"] in (1, 2, 4, 8, 16) and 0 < t["block_pairs"] <= 8192 and t["us_per_pair"] > 0
        assert t["cta_pair"] in (0, 1)
        # the tuned plan still computes Eq. 1
        rng = np.random.default_rng(2)
        M = (rng.standard_normal((4 * 40, 350)) + 1j * rng.standard_normal((4 * 40, 350))) * 0.02
        Ev, Ec = prob.E_v[:4], prob.E_c[:40]
        dE = (Ev[:, None] - Ec[None, :]).reshape(-1)
        ref = chi0_from_pairs(M, freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta))
        chi = plan.accumulate(0, _dev(M.astype(np.complex64)), 4, 40, _dev(Ev), _dev(Ec)).cpu().numpy()
        assert max(rel_fro(chi[i], ref[i]) for i in range(3)) < TOL
    lines = (tmp_path / "tune.txt").read_text().splitlines()
    assert len(lines) == 1 and f"group={t['group']}" in lines[0]
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp16", max_pairs=8192) as plan2:
        t2 = plan2.autotune(0)          # served from the cache
        assert t2["us_per_pair"] == -1.0
        assert (t2["group"], t2["block_pairs"], t2["cta_pair"]) == (t["group"], t["block_pairs"], t["cta_pair"])
