"""Allocation-free misfit entry point (gsw_misfit_noalloc) against gsw_misfit_green.

Some callers cannot allocate GPU memory: their device memory is owned by
another allocator (a framework's caching pool or an arena reserved at start-up)
or they run in a loop where cudaMalloc/cudaFree would synchronise the device.
For them the library keeps this variant's working memory in one fixed
device array.  The test feeds it caller-owned device buffers through the C
ABI and checks it against the allocating entry point, on two calls in a row
(the second call must not see the first call's leftovers), with the same
tolerances as the misfit parity test.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _problem(seed, n_rec=6, n_t=240, s=6, L=12):
    rng = np.random.default_rng(seed)
    t = np.arange(n_t)
    G = np.zeros((n_rec, 3, 3, n_t))
    for k in range(n_rec):
        for i in range(3):
            for j in range(3):
                G[k, i, j] = rng.standard_normal() * np.sin(2 * np.pi * rng.uniform(0.01, 0.08) * t) * np.exp(-t / 80)
    obs = rng.standard_normal((n_rec, 3, n_t))
    obs[1, 2] = 0.0
    return G, obs, s, L


def test_noalloc_misfit_matches_allocating_entry_point():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_17754_gb300 import build, gsw

    build.build()
    ctx = gsw.Context(0)
    try:
        for seed in (21, 22):  # two calls in a row with different data
            G, obs, s, L = _problem(seed)
            e_ref, c_ref = ctx.misfit_green(G, obs, s, L, tau=1e-10)
            G_dev = torch.tensor(G, device="cuda")
            obs_dev = torch.tensor(obs, device="cuda")
            err_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            c_dev = torch.full((3, L), float("nan"), dtype=torch.float64, device="cuda")
            ctx.misfit_noalloc(G_dev, obs_dev, s, L, err_dev, c_dev, tau=1e-10)
            torch.cuda.synchronize()
            e = float(err_dev.cpu()[0])
            c = c_dev.cpu().numpy()
            assert abs(e - e_ref) <= 1e-9 * e_ref
            assert np.abs(c - c_ref).max() <= 1e-8 * np.abs(c_ref).max()
        # sizes beyond the fixed working memory are rejected
        G, obs, s, _ = _problem(23, n_rec=2, n_t=100)
        G_dev = torch.tensor(G, device="cuda")
        obs_dev = torch.tensor(obs, device="cuda")
        err_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(gsw.GswError) as ei:
            ctx.misfit_noalloc(G_dev, obs_dev, 1, 65, err_dev)
        assert ei.value.status == gsw.E_INVALID
        G, obs, s, L = _problem(24, n_rec=1025, n_t=16, L=2)
        with pytest.raises(gsw.GswError) as ei:
            ctx.misfit_noalloc(torch.tensor(G, device="cuda"), torch.tensor(obs, device="cuda"), s, L, err_dev)
        assert ei.value.status == gsw.E_INVALID
        # the input-wave coefficients are optional
        G, obs, s, L = _problem(25)
        e_ref, _ = ctx.misfit_green(G, obs, s, L, tau=1e-10)
        err_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.misfit_noalloc(torch.tensor(G, device="cuda"), torch.tensor(obs, device="cuda"), s, L, err_dev, None)
        torch.cuda.synchronize()
        assert abs(float(err_dev.cpu()[0]) - e_ref) <= 1e-9 * e_ref
        # outputs smaller than the result are refused before any launch
        with pytest.raises(ValueError):
            ctx.misfit_noalloc(torch.tensor(G, device="cuda"), torch.tensor(obs, device="cuda"), s, L, err_dev,
                               torch.zeros(3 * L - 1, dtype=torch.float64, device="cuda"))
    finally:
        ctx.close()
