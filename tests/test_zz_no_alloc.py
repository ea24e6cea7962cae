"""blaz_dot_noalloc, the flattened dot product for callers that cannot let
the library allocate device memory (a framework or server owning all of HBM,
a device without stream-ordered allocation, a step that must not risk an
allocation failure).  It keeps its scratch in a fixed array inside the
library and launches the same kernel on the same grid as blaz_dot, so this
test checks, through the C ABI, that two calls in a row (the second finds
the first call's leftovers in that array) return blaz_dot's bits, and that
both stay within the dot tolerance, 1e-12 * sum |A_hat B_hat|, of the
oracle.  The 4096^2 pair launches the largest grid (min(6 x SMs, 1024)
CTAs), so every partial-sum slot a GB300 uses is written and read back.

The file is named to be collected last; it passes alone in a fresh process
and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot_on_two_calls_in_a_row():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    L = blaz.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    A, B = W.plain_pair()
    pairs = [(A, B), (W.bump_field(1024, 1024), W.bump_field(1024, 1025)),
             (W.bump_field(4096, 4096), W.bump_field(4096, 4097))]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for X, Y in pairs:
        ga = blaz.compress(torch.from_numpy(X).to(dev))
        gb = blaz.compress(torch.from_numpy(Y).to(dev))
        want = blaz.dot(ga, gb)
        ref, abs_sum = O.dot(O.compress(X), O.compress(Y))
        da, db = ga.desc(), gb.desc()
        for _ in range(2):
            out = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
            rc = L.blaz_dot_noalloc(ctypes.byref(da), ctypes.byref(db), out.data_ptr(), stream)
            assert rc == 0, L.blaz_strerror(rc)
            assert torch.equal(out, want.reshape(1))
            assert abs(float(out.item()) - ref) <= 1e-12 * abs_sum
