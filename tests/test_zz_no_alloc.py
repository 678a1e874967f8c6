"""The allocation-free host-buffer call (sph_filter_apply_host_noalloc), through the C ABI (GPU).

It serves callers that cannot let the library allocate device memory: its device staging is a
fixed array inside the library. Its results must equal those of sph_filter_apply_host, which uses
staging buffers the plan allocates, on consecutive calls (the array keeps the previous call's
contents), and states beyond its capacity must be refused. This file is collected last so that a
run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_2305_01537_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


def _errors(y, ref):
    return max(np.abs(y[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300) for v in range(ref.shape[0]))


def test_noalloc_matches_allocating_call_twice(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan, binding
    lib = binding.load()
    for prec in (0, 2, 1, 3):  # FP64, compensated FP32, split-precision tensor-core form, spectral form
        g = W.grid_28(8, 32, 64)  # 458,752 points, within the 2,097,152-point capacity
        g.r = np.linspace(0.5, 30.5, 8)
        plan = Plan.from_grid(g, precision=prec)
        stream = torch.cuda.current_stream()
        for seed in (11, 12):  # two calls in a row, different data
            x = torch.from_numpy(W.band_limited_state(g, seed=seed, mode_max=6, noise=0.05)).pin_memory()
            ref = torch.empty_like(x).pin_memory()
            got = torch.empty_like(x).pin_memory()
            plan.apply_host(x, ref)
            st = lib.sph_filter_apply_host_noalloc(plan._h, x.data_ptr(), got.data_ptr(), stream.cuda_stream)
            assert st == 0
            torch.cuda.synchronize()
            assert plan.sync_status() == 0
            # the tensor-core form's tolerance against the oracle is 1e-11; the two calls run the same
            # kernels on the same data and must agree far closer than that
            assert _errors(got.numpy(), ref.numpy()) <= TOL


def test_noalloc_rejects_states_beyond_capacity(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan, binding
    lib = binding.load()
    g = W.grid_28(48, 32, 64)  # 2,752,512 points > 2,097,152
    plan = Plan.from_grid(g)
    x = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
    out = torch.zeros_like(x).pin_memory()
    st = lib.sph_filter_apply_host_noalloc(plan._h, x.data_ptr(), out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert st == binding.SPH_EINVAL
