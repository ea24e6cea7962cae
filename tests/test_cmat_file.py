"""Compressed-matrix files (save / load of the Sec. II block payload).

The CPU tests write files from the layout documented in include/blaz.h with
plain Python (an independent writer) and check that the library reads the
shape back and rejects every malformed variant before touching a device.
The GPU tests round-trip compressed matrices through files and load files
written by Python from the oracle's compression."""
import ctypes
import os
import struct

import numpy as np
import pytest

import oracle as O
import workloads as W

NKEEP = 28


def fnv1a(data: bytes) -> int:
    """FNV-1a 64 over little-endian 64-bit words, the last one zero-padded."""
    h = 14695981039346656037
    data = data + b"\0" * (-len(data) % 8)
    for (w,) in struct.iter_unpack("<Q", data):
        h ^= w
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def file_bytes(rows, cols, f, s, phi, code, *, magic=b"BLAZCMAT", version=1, hbytes=64, nb=None,
               pbytes=None, hash_=None, zero=0):
    nbk = (rows // 8) * (cols // 8)
    payload = (np.asarray(f, "<f8").tobytes() + np.asarray(s, "<f8").tobytes() +
               np.asarray(phi, np.uint8).tobytes() + np.asarray(code, np.int8).tobytes())
    head = magic + struct.pack("<IIqqqQQQ", version, hbytes, rows, cols, nbk if nb is None else nb,
                               len(payload) if pbytes is None else pbytes,
                               fnv1a(payload) if hash_ is None else hash_, zero)
    assert len(head) == 64
    return head + payload


def oracle_payload(A):
    c = O.compress(A)
    return c.f, c.s, c.phi, c.code


@pytest.fixture(scope="module")
def L():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    return blaz


def _info(L, path):
    r, c = ctypes.c_int64(), ctypes.c_int64()
    rc = L.lib().blaz_cmat_file_info(os.fsencode(path), ctypes.byref(r), ctypes.byref(c))
    return rc, r.value, c.value


def _load_status(L, path, rows, cols):
    d = L._CMatDesc(rows, cols, 0, 0, 0, 0)
    return L.lib().blaz_cmat_load(os.fsencode(path), ctypes.byref(d), None)


def test_file_info_reads_the_documented_layout(L, tmp_path):
    A = W.random_block_matrix(16, 24, seed=1)
    p = tmp_path / "a.blaz"
    p.write_bytes(file_bytes(16, 24, *oracle_payload(A)))
    assert _info(L, p) == (0, 16, 24)
    q = tmp_path / "empty.blaz"
    q.write_bytes(file_bytes(0, 8, [], [], [], np.zeros((0, NKEEP), np.int8)))
    assert _info(L, q) == (0, 0, 8)


def test_malformed_files_are_rejected_before_any_device_access(L, tmp_path):
    A = W.random_block_matrix(16, 24, seed=2)
    pl = oracle_payload(A)
    good = file_bytes(16, 24, *pl)
    variants = {
        "magic": file_bytes(16, 24, *pl, magic=b"BLAZCMAX"),
        "version": file_bytes(16, 24, *pl, version=2),
        "header": file_bytes(16, 24, *pl, hbytes=72),
        "nb": file_bytes(16, 24, *pl, nb=5),
        "payload": file_bytes(16, 24, *pl, pbytes=45 * 6 + 1),
        "shape": file_bytes(12, 24, *pl, nb=6),
        "zero": file_bytes(16, 24, *pl, zero=1),
        "truncated": good[:-1],
        "trailing": good + b"\0",
        "hash": good[:-1] + bytes([good[-1] ^ 1]),
    }
    FORMAT, IO, SHAPE = -12, -11, -1
    for name, data in variants.items():
        p = tmp_path / f"{name}.blaz"
        p.write_bytes(data)
        if name in ("truncated", "trailing", "hash"):
            assert _info(L, p)[0] == 0, name            # the header alone is fine
        else:
            assert _info(L, p)[0] == FORMAT, name
        assert _load_status(L, p, 16, 24) == FORMAT, name
    p = tmp_path / "good.blaz"
    p.write_bytes(good)
    assert _load_status(L, p, 16, 32) == SHAPE          # caller's matrix has another shape
    assert _info(L, tmp_path / "missing.blaz")[0] == IO
    assert _load_status(L, tmp_path / "missing.blaz", 16, 24) == IO


@pytest.mark.gpu
def test_round_trip_is_bit_exact(L, tmp_path):
    import torch

    for shape, seed in (((64, 136), 3), ((8, 8), 4), ((0, 16), 5), ((1024, 520), 6)):
        A = W.random_block_matrix(*shape, seed=seed) if shape[0] else np.zeros(shape)
        g = L.compress(torch.from_numpy(A).cuda())
        p = tmp_path / f"m{seed}.blaz"
        L.save(g, p)
        assert L.file_info(p) == shape
        h = L.load(p)
        for x, y in zip(g.to_host(), h.to_host()):
            assert x.tobytes() == y.tobytes()


@pytest.mark.gpu
def test_loads_a_file_written_from_the_oracle(L, tmp_path):
    A = W.random_block_matrix(72, 64, seed=7, kind="noise")
    f, s, phi, code = oracle_payload(A)
    p = tmp_path / "oracle.blaz"
    p.write_bytes(file_bytes(72, 64, f, s, phi, code))
    h = L.load(p)
    gf, gs, gphi, gcode = h.to_host()
    assert gf.tobytes() == f.tobytes() and gs.tobytes() == s.tobytes()
    assert np.array_equal(gphi, phi) and np.array_equal(gcode, code)
    # and the library saves the same bytes back
    q = tmp_path / "again.blaz"
    L.save(h, q)
    assert q.read_bytes() == p.read_bytes()
