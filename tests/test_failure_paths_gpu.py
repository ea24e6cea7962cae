"""Failure paths on the GPU, produced without faulting it: a bounded device
wait that runs out (a flag nothing sets) reports BLAZ_ERR_TIMEOUT through the
device status word and leaves the context usable; an allocation the device
cannot satisfy reports BLAZ_ERR_OOM; outputs never write outside their
arrays (guard bands around every array of a compressed matrix)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TIMEOUT, OOM, SHAPE = -7, -4, -1


@pytest.fixture(scope="module")
def B():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    blaz.lib()
    torch.cuda.init()
    return blaz


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_bounded_wait_runs_out_and_the_context_stays_usable(B):
    assert B.device_status() == 0
    assert B.lib().blaz_probe_bounded_wait(100_000_000, _stream()) == 0   # ~50 ms at 2 GHz
    assert B.device_status() == TIMEOUT
    assert B.device_status() == 0                                        # read and cleared
    A = W.random_block_matrix(64, 72, seed=3)
    g = B.compress(torch.from_numpy(A).cuda())
    o = O.compress(A)
    assert np.array_equal(g.code.cpu().numpy(), o.code)


def test_allocation_failure_is_reported(B):
    d = B._CMatDesc(0, 0, 0, 0, 0, 0)
    side = 1 << 23                                                       # 2^40 blocks, 49 TB
    assert B.lib().blaz_cmat_alloc(ctypes.byref(d), side, side, _stream()) == OOM
    assert B.lib().blaz_cmat_alloc(ctypes.byref(d), 1 << 35, 8, _stream()) == SHAPE
    # the device is still fine
    g = B.compress(torch.zeros((16, 16), dtype=torch.float64, device="cuda"))
    assert g.nb == 4


def test_outputs_stay_inside_their_arrays(B):
    """Compressed outputs written into views of larger buffers filled with a
    sentinel: only the views change (compress, add, scale, load)."""
    rows, cols = 72, 136
    nb = (rows // 8) * (cols // 8)
    pad = 64
    store = [torch.full((nb + 2 * pad,), 7.25, dtype=torch.float64, device="cuda") for _ in range(2)]
    store += [torch.full((nb + 2 * pad,), 0xA5, dtype=torch.uint8, device="cuda"),
              torch.full((nb + 2 * pad, 28), 90, dtype=torch.int8, device="cuda")]
    out = B.CMat(rows, cols, store[0][pad:pad + nb], store[1][pad:pad + nb], store[2][pad:pad + nb],
                 store[3][pad:pad + nb])

    def guards_intact():
        for t in store:
            head, tail = t[:pad].cpu().numpy(), t[pad + nb:].cpu().numpy()
            ref = t.view(-1)[0].item()
            assert np.all(head == ref) and np.all(tail == ref)

    A = W.random_block_matrix(rows, cols, seed=11, kind="noise")
    Bm = W.random_block_matrix(rows, cols, seed=12)
    B.compress(torch.from_numpy(A).cuda(), out=out)
    guards_intact()
    gb = B.compress(torch.from_numpy(Bm).cuda())
    B.add(out, gb, out=out)
    guards_intact()
    B.scale(out, -3.0, out=out)
    guards_intact()
    ref = O.scale(O.add(O.compress(A), O.compress(Bm)), -3.0)
    assert np.array_equal(out.code.cpu().numpy(), ref.code)


def test_fp64_probe_counts_its_additions(B):
    """The binary64 issue-rate probe launches 4 additions per thread and round
    on one CTA of 32 w threads per SM, and its rate is a positive number."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(sms * 16 * 32, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    ops = B.probe_fp64_rate(256, out, 16, st)
    e1.record(st)
    torch.cuda.synchronize()
    assert ops == sms * 16 * 32 * 256 * 4
    assert ops / (e0.elapsed_time(e1) * 1e-3) > 1e9
    # each thread's 4 chains start at tid * 1e-3 + i and add 256 ones each
    t = torch.arange(16 * 32, dtype=torch.float64, device="cuda") * 1e-3
    assert torch.allclose(out[: 16 * 32], 4 * t + (0 + 1 + 2 + 3) + 4 * 256.0, rtol=1e-12, atol=0)
    with pytest.raises(B.BlazError):
        B.probe_fp64_rate(256, out[:10], 16, st)
