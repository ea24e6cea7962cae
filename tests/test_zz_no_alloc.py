"""blaz_dot_noalloc, the flattened dot product for callers that cannot let
the library allocate device memory (a framework or server owning all of HBM,
a device without stream-ordered allocation, a step that must not risk an
allocation failure).  It keeps its scratch in a fixed array inside the
library, so this test checks, through the C ABI, that two calls in a row
(the second finds the first call's leftovers in that array) give the same
result as blaz_dot within the dot tolerance, 1e-12 * sum |A_hat B_hat|.

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
    F, G = W.bump_field(1024, 1024), W.bump_field(1024, 1025)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for X, Y in [(A, B), (F, G)]:
        ga = blaz.compress(torch.from_numpy(X).to(dev))
        gb = blaz.compress(torch.from_numpy(Y).to(dev))
        want = float(blaz.dot(ga, gb).item())
        _, abs_sum = O.dot(O.compress(X), O.compress(Y))
        da, db = ga.desc(), gb.desc()
        for _ in range(2):
            out = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
            rc = L.blaz_dot_noalloc(ctypes.byref(da), ctypes.byref(db), out.data_ptr(), stream)
            assert rc == 0, blaz.lib().blaz_strerror(rc)
            got = float(out.item())
            assert abs(got - want) <= 1e-12 * abs_sum
