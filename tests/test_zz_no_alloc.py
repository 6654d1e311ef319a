"""The allocation-free first-region test against the enumeration's own test.

gc_fp_test_static serves callers that cannot allocate device memory (graph
capture, fixed memory budgets, caller-owned arenas): it keeps its scratch in a
fixed device array.  This file is collected last so that, in a run that stops
at the first failure, every other test has already run; it also passes alone
in a fresh process, where its first call performs the per-device set-up.
"""
import numpy as np
import pytest

import orbit_inputs as oi
from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu

CASES = [(3, 4, 0.7, 12), (2, 6, 1.0, 5)]   # two different lattices, one call each


def test_static_fp_test_matches_enumeration_twice():
    import torch
    import paper_1403_0555_b300 as gb

    torch.cuda.init()
    stream = torch.cuda.current_stream()
    for d, L, kappa, seed in CASES:
        V = L ** d
        phi = oi.von_mises_orbit(d, L, kappa, seed)
        # reference: the enumeration's dense Faddeev-Popov test (existing entry point)
        _, ref, _ = run_gpu(d, L, phi, seed, 1500, keep_per_start=0, fp_mode=gb.GC_FP_DENSE)
        n = ref["n_distinct"]
        assert n > 1
        links = torch.tensor(np.stack([np.cos(phi), np.sin(phi)], axis=-1).reshape(-1, 2),
                             dtype=torch.float64, device="cuda")
        cfg = torch.tensor(np.stack([np.cos(ref["theta"]), np.sin(ref["theta"])], axis=-1),
                           dtype=torch.float64, device="cuda")
        lam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        reg = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        gb.gc_fp_test_static(d, L, links.data_ptr(), cfg.data_ptr(), n, 1e-9, lam.data_ptr(),
                             reg.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        lam_h = lam.cpu().numpy()
        reg_h = reg.cpu().numpy()
        assert np.max(np.abs(lam_h - ref["lambda2"])) < 1e-9
        assert np.array_equal(reg_h, ref["region"])


def test_static_fp_test_rejects_oversized_requests():
    import paper_1403_0555_b300 as gb
    with pytest.raises(gb.GribovError) as e:
        gb.gc_fp_test_static(2, 4, 1, 1, (1 << 16) + 1, 1e-9, 1, 1, 0)
    assert e.value.code == gb.GC_EINVAL and "per-call maximum" in gb.gc_last_error()
    with pytest.raises(gb.GribovError) as e:
        gb.gc_fp_test_static(4, 8, 1, 1, 4, 1e-9, 1, 1, 0)      # 4096 sites: basis too large
    assert e.value.code == gb.GC_EINVAL and "static scratch" in gb.gc_last_error()
