"""Host buffers: compression of a matrix in host memory (transfer pipelined
with compression through a ring of staging buffers) and the packed payload
to / from host memory.  The host path must give the bits of the device path
and of the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    blaz.lib()
    torch.cuda.init()
    return blaz


def same(g, h):
    for x, y in zip(g.to_host(), h.to_host()):
        assert x.tobytes() == y.tobytes()


# (rows, cols): one slab; six slabs of 16 rows (128 MB each) and a ragged
# last one of 8 rows (the ring of 4 staging buffers is reused); slabs of 16,
# 16 and 8 rows
@pytest.mark.parametrize("shape", [(72, 136), (88, 1048576), (40, 786432)])
def test_compress_from_pinned_host_memory(B, shape):
    rows, cols = shape
    t = W.bump_field_torch(cols, rows + cols, "cuda", rows=rows)
    h = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    h.copy_(t)
    torch.cuda.synchronize()
    g = B.compress_host(h)
    torch.cuda.synchronize()
    assert B.device_status() == 0
    same(g, B.compress(t))
    # sampled blocks against the oracle
    nbc = cols // 8
    rng = np.random.default_rng(rows)
    idx = np.unique(np.concatenate([rng.integers(0, g.nb, 200), [0, g.nb - 1]]))
    hn = h.numpy()
    blocks = np.concatenate([hn[8 * (b // nbc):8 * (b // nbc) + 8, 8 * (b % nbc):8 * (b % nbc) + 8] for b in idx])
    o = O.compress(blocks)
    f, s, phi, code = g.to_host()
    assert np.array_equal(code[idx], o.code) and np.array_equal(phi[idx], o.phi)
    assert f[idx].tobytes() == o.f.tobytes() and s[idx].tobytes() == o.s.tobytes()


def test_compress_from_pageable_memory_and_strided_rows(B):
    A = W.random_block_matrix(64, 200, seed=4)
    h = torch.from_numpy(A)                       # pageable
    g = B.compress_host(h[:, 8:192])              # lda = 200
    torch.cuda.synchronize()
    same(g, B.compress(torch.from_numpy(np.ascontiguousarray(A[:, 8:192])).cuda()))


def test_payload_download_upload_round_trip(B):
    A = W.random_block_matrix(48, 104, seed=5, kind="noise")
    g = B.compress(torch.from_numpy(A).cuda())
    host = torch.empty(g.nbytes, dtype=torch.uint8, pin_memory=True)
    B.download(g, host)
    torch.cuda.synchronize()
    f, s, phi, code = g.to_host()
    want = f.tobytes() + s.tobytes() + phi.tobytes() + code.tobytes()   # the file payload layout
    assert host.numpy().tobytes() == want
    h2 = B.CMat.empty(48, 104)
    B.upload(host, h2)
    torch.cuda.synchronize()
    same(g, h2)


def test_host_entry_point_errors(B):
    import ctypes

    h = torch.zeros((16, 24), dtype=torch.float64)
    out = B.CMat.empty(16, 24)
    d = out.desc()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert B.lib().blaz_compress_host(ctypes.c_void_p(h.data_ptr()), 23, ctypes.byref(d), st) == -3
    assert B.lib().blaz_compress_host(None, 24, ctypes.byref(d), st) == -2
    assert B.lib().blaz_cmat_download(ctypes.byref(d), None, st) == -2


def test_back_to_back_calls_reuse_the_staging_ring(B):
    """The staging ring persists from call to call: calls of different slab
    sizes issued back to back, alternating between two streams and with no
    synchronization between them, each give the device path's bits (a
    buffer is refilled only after the compression of its previous slab)."""
    shapes = [(88, 786432), (72, 136), (40, 327680), (88, 786432), (16, 1048576), (72, 136)]
    srcs, outs = [], []
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k, (rows, cols) in enumerate(shapes):
        t = W.bump_field_torch(cols, 7 * k + rows, "cuda", rows=rows)
        h = torch.empty((rows, cols), dtype=torch.float64, pin_memory=True)
        h.copy_(t)
        srcs.append((t, h))
    torch.cuda.synchronize()
    for k, (t, h) in enumerate(srcs):
        st = streams[k % 2]
        with torch.cuda.stream(st):
            outs.append(B.compress_host(h, stream=st))
    torch.cuda.synchronize()
    assert B.device_status() == 0
    for (t, h), g in zip(srcs, outs):
        same(g, B.compress(t))
