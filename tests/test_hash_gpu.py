"""Parity of the hash scans (SHA256 / Blake256 / Blake2B, Sec. 4.1) with the
oracle, alone and horizontally fused: digests bit for bit, hit sets exactly."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import DEV, single  # noqa: E402
from paper_2007_01277_gb300 import hfuse as H  # noqa: E402
from paper_2007_01277_gb300 import workloads as W  # noqa: E402

SCAN = {H.SHA256D: oracle.sha256d_scan, H.BLAKE256: oracle.blake256_scan,
        H.BLAKE2B: oracle.blake2b_scan}
HASHES = list(SCAN)


class Scan:
    """Device buffers and the argument block of one scan."""

    def __init__(self, body, header, first, n, target=0, cap=0, digests=True):
        self.body, self.header, self.first, self.n, self.target = body, header, first, n, target
        self.dig = torch.zeros(max(n, 1) * 32, dtype=torch.uint8, device=DEV) if digests else None
        self.hits = torch.full((cap,), -1, dtype=torch.int32, device=DEV) if cap else None
        self.cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
        self.args = H.hash_scan_args(header, n, first, target, self.dig, self.hits, self.cnt)

    def ref(self):
        return SCAN[self.body](self.header, self.first, self.n)

    def check(self):
        ref = self.ref()
        if self.dig is not None:
            got = self.dig[: 32 * self.n].cpu().numpy().reshape(self.n, 32)
            assert np.array_equal(got, ref), H.BODY_NAMES[self.body]
        want = oracle.hash_hits(ref, self.first, self.target)
        assert int(self.cnt.item()) == want.size
        if self.hits is not None:
            got = self.hits.cpu().numpy().view(np.uint32)[: min(want.size, self.hits.numel())]
            if want.size <= self.hits.numel():
                assert np.array_equal(np.sort(got), want)
            else:   # capacity exceeded: every stored nonce is a hit, none twice
                assert np.unique(got).size == got.size and np.isin(got, want).all()


@pytest.mark.parametrize("body", HASHES)
@pytest.mark.parametrize("n,threads,grid,first", [(5003, 128, 7, 0), (1, 32, 1, 123),
                                                  (4133, 256, 19, 0xFFFFFF00), (700, 96, 3, 99)])
def test_scan_digests_and_hits(body, n, threads, grid, first):
    s = Scan(body, W.hash_header(1), first, n, target=1 << 28, cap=n)
    single(body, s.args, threads, grid)
    torch.cuda.synchronize()
    s.check()


@pytest.mark.parametrize("body", HASHES)
def test_scan_hits_only_and_capacity(body):
    # no digest buffer (the mining mode); one nonce in 64 hits
    s = Scan(body, W.hash_header(2), 1000, 20000, target=1 << 26, cap=4096, digests=False)
    single(body, s.args, 256, 40)
    torch.cuda.synchronize()
    s.check()
    # capacity below the number of hits: all hits counted, cap of them stored
    s = Scan(body, W.hash_header(2), 1000, 20000, target=1 << 26, cap=50, digests=False)
    single(body, s.args, 256, 40)
    torch.cuda.synchronize()
    s.check()
    assert (s.hits.cpu() != -1).all()


@pytest.mark.parametrize("body", HASHES)
def test_scan_empty_and_invalid(body):
    s = Scan(body, W.hash_header(3), 0, 0, target=0xFFFFFFFF, cap=4)
    single(body, s.args, 64, 2)
    torch.cuda.synchronize()
    assert int(s.cnt.item()) == 0 and (s.hits.cpu() == -1).all()
    k = H.hf_register_kernel(body)
    bad = H.hash_scan_args(W.hash_header(3), 10, hit_count=s.cnt)
    bad.hit_cap = 5   # capacity without a hits buffer
    with pytest.raises(H.HFError):
        H.hf_launch_single(k, bad, 64, 1)
    bad = H.hash_scan_args(W.hash_header(3), -1)
    with pytest.raises(H.HFError):
        H.hf_launch_single(k, bad, 64, 1)


PAIRS = [(H.SHA256D, H.BLAKE256), (H.SHA256D, H.BLAKE2B), (H.BLAKE256, H.BLAKE2B)]


@pytest.mark.parametrize("a,b", PAIRS)
@pytest.mark.parametrize("split,d0,cap,grid", [(128, 256, 0, 11), (64, 512, 64, 5), (384, 512, 40, 3)])
def test_fused_hash_pairs(a, b, split, d0, cap, grid):
    sa = Scan(a, W.hash_header(4), 0, 3001, target=1 << 27, cap=512)
    sb = Scan(b, W.hash_header(5), 17, 2999, target=1 << 27, cap=512)
    f = H.hf_fuse(H.hf_register_kernel(a), H.hf_register_kernel(b), split, d0, cap)
    H.hf_launch(f, [sa.args, sb.args], grid)
    torch.cuda.synchronize()
    sa.check()
    sb.check()
    # bit-exact to the standalone launches at the same interval size and grid
    for s, thr in ((sa, split), (sb, d0 - split)):
        t = Scan(s.body, s.header, s.first, s.n, s.target, cap=512)
        single(s.body, t.args, thr, grid)
        torch.cuda.synchronize()
        assert torch.equal(t.dig, s.dig)


def test_hash_with_memory_kernel_and_nway():
    # a compute-bound hash next to a memory-bound kernel (no compiled pair:
    # the N-way instance), and all three hashes in one N-way launch
    sh = Scan(H.SHA256D, W.hash_header(6), 5, 2048, target=1 << 28, cap=256)
    x = W.upsample_input((3, 5, 17, 20))
    y = torch.empty(3, 5, 34, 40, device=DEV)
    f = H.hf_fuse(H.hf_register_kernel(H.SHA256D), H.hf_register_kernel(H.UPSAMPLE2X), 128, 256, 0)
    H.hf_launch(f, [sh.args, H.upsample2x_args(x.to(DEV), y)], 6)
    torch.cuda.synchronize()
    sh.check()
    ref = oracle.upsample2x(x.numpy())
    assert np.allclose(y.double().cpu().numpy(), ref, rtol=1e-5, atol=0)
    scans = [Scan(b, W.hash_header(7 + i), 100 * i, 1500 + i, target=1 << 27, cap=256)
             for i, b in enumerate(HASHES)]
    ks = [H.hf_register_kernel(b) for b in HASHES]
    # sha256d and blake256 share interval 0 (run one after the other)
    f = H.hf_fuse_n(ks, [0, 0, 1], [128, 64], 0)
    H.hf_launch(f, [s.args for s in scans], 4)
    torch.cuda.synchronize()
    for s in scans:
        s.check()
