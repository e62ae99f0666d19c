"""The allocation-free batch-norm entry point against the workspace one.

hf_bn_stats_noalloc serves callers that must not allocate device memory; its
scratch is a fixed device array inside the library.  This file is collected
last on purpose.  The test calls the new entry point through the C ABI
twice in a row on the same inputs (the second call must find the shared
array usable again), then once on another shape, and compares each result
with hf_launch_single of the batch-norm body using a caller workspace at the
same threads and grid: both run the same body and combine each channel's
tile sums in tile order, so the results must agree bit for bit; each result
is also checked against the oracle under the tolerance the other batch-norm
tests use, and the device error word must stay clear.  It also checks that a
shape too large for the fixed array is rejected.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import DEV, check_bn  # noqa: E402
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402


def _reference(xd, threads, grid):
    C = xd.shape[1]
    mean, var = torch.empty(C, device=DEV), torch.empty(C, device=DEV)
    k = H.hf_register_kernel(H.BN_STATS)
    H.hf_launch_single(k, H.bn_stats_args(xd, mean, var, H.bn_stats_workspace(xd)), threads, grid)
    torch.cuda.synchronize()
    H.hf_destroy_kernel(k)
    return mean, var


def _same(x_cpu, m, v, m_ref, v_ref):
    assert torch.equal(m, m_ref) and torch.equal(v, v_ref)
    check_bn(x_cpu, m, v)


@pytest.mark.parametrize("threads,grid", [(256, 0), (128, 37)])
def test_noalloc_matches_workspace_entry_point(threads, grid):
    x = W.bn_input((8, 64, 32, 32), seed=3)
    xd = x.to(DEV)
    m_ref, v_ref = _reference(xd, threads, grid)
    for _ in range(2):   # two calls in a row share the fixed scratch array
        m = torch.full((64,), float("nan"), device=DEV)
        v = torch.full((64,), float("nan"), device=DEV)
        H.hf_bn_stats_noalloc(xd, m, v, threads, grid)
        torch.cuda.synchronize()
        assert H.hf_check_device_error() == 0
        _same(x, m, v, m_ref, v_ref)
    # another shape (more channels, a ragged last tile) after the first two
    x2 = W.bn_input((5, 96, 17, 20), seed=4)
    x2d = x2.to(DEV)
    m2_ref, v2_ref = _reference(x2d, threads, grid)
    m2, v2 = torch.empty(96, device=DEV), torch.empty(96, device=DEV)
    H.hf_bn_stats_noalloc(x2d, m2, v2, threads, grid)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    _same(x2, m2, v2, m2_ref, v2_ref)


def test_noalloc_rejects_shapes_beyond_the_fixed_array():
    # 64 channels of 2^22 values need 64 * 2048 tiles * 8 bytes = 1 MiB of
    # partial sums plus 256 bytes of counters: more than the fixed array.
    # The shape is checked on the host before anything is queued, so a small
    # buffer stands in for the (never read) 1 GiB input.
    buf = torch.zeros(64, device=DEV)
    p = buf.data_ptr()
    st = H.lib.hf_bn_stats_noalloc(p, p, p, 1, 64, 1 << 22, 256, 0,
                                   torch.cuda.current_stream().cuda_stream)
    assert st == -1 and b"scratch" in H.lib.hf_last_error()
    # a small shape goes through on the same array right after the refusal
    x = torch.tensor([[[[1.0, 2.0, 3.0, 4.0]]]], device=DEV)
    m, v = torch.empty(1, device=DEV), torch.empty(1, device=DEV)
    H.hf_bn_stats_noalloc(x, m, v, 256, 1)
    torch.cuda.synchronize()
    assert H.hf_check_device_error() == 0
    assert m.item() == 2.5 and v.item() == 1.25
