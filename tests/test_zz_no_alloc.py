"""The allocation-free mu search (tb_find_mu_static) against the context-based
one (tb_find_mu) on the same spectral record, through the C ABI.

Callers that may not allocate device memory (a host runtime owning every
device allocation through its own pool) use tb_find_mu_static: it needs no
tb_ctx and keeps its scratch in a fixed array inside the library.  It must
give the same chemical potential as tb_find_mu, on every call: the array
keeps the previous call's contents, so two calls run back to back here, and
the second call (after the one-time set-up) must leave the device's free
memory and torch's allocation count unchanged.

This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from synth import CONFIGS, fcc_c60_crystal, workload_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_mu_matches_context_mu_twice(tb, prec):
    cfg = CONFIGS[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    s.evaluate()                      # lists, H, spectral record, tb_find_mu, forces
    torch.cuda.synchronize()
    s.check()
    mu_ref = s.mu.item()
    n_ref = s.ncount.item()
    ne = 4.0 * s.n
    outs = [(torch.full((1,), float("nan"), dtype=torch.float64, device="cuda"),
             torch.zeros(1, dtype=torch.float64, device="cuda"),
             torch.full((2,), -7, dtype=torch.int32, device="cuda")) for _ in range(2)]
    for call, (mu, ncount, status) in enumerate(outs):
        if call == 1:
            # the first call did the one-time set-up: from here on nothing may
            # allocate, neither on the device nor through torch's allocator
            free0 = torch.cuda.mem_get_info()[0]
            allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        tb.binding.tb_find_mu_static(s.n, s.tp.r, s.lam, s.S, p["kT"], ne, s.tp.mu_tol,
                                     s.tp.mu_max_iter, None, mu, ncount, status)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
        assert status.tolist() == [0, 0], f"call {call}: device status {status.tolist()}"
        # same search on the same data and grid: the electron count tolerance of
        # the parity tests, and in practice the same bits
        assert abs(ncount.item() - ne) <= 1e-9 * s.n
        assert abs(mu.item() - mu_ref) <= 1e-9
        assert abs(ncount.item() - n_ref) <= 1e-9 * s.n
    s.close()


def test_static_mu_rejects_bad_arguments(tb):
    from paper_0910_4497_gb300.binding import TBError
    lam = torch.zeros(32, dtype=torch.float64, device="cuda")
    S = torch.zeros(4 * 32, dtype=torch.float64, device="cuda")
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(TBError) as e:
        tb.binding.tb_find_mu_static(1, 17, lam, S, 0.1, 4.0, 1e-12, 100, None, mu, None, status)
    assert e.value.code == 1
    with pytest.raises(TBError):
        tb.binding.tb_find_mu_static(1, 8, lam, S, 0.1, 4.0, 1e-12, 100, None, mu, None, None)
