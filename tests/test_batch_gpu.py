"""Batched mixed operations (one persistent, graph-captured launch).

Every result of a batch must equal the same operation run alone: bit for bit
for compress / add / sub / scale (same device code), within the dot and
product tolerances otherwise.  Small batches are also checked against the
oracle directly; the full batch workload (2000 ops, sides 64..2048) is
checked on sampled operations."""
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
    return blaz


def _field(rows, cols, seed):
    return W.bump_field_torch(cols, seed, "cuda", rows=rows)


def make_batch(B, specs, with_decompress=True):
    """Inputs and outputs for a list of workload op descriptors."""
    ops, meta = [], []
    for i, d in enumerate(specs):
        r, c, seed = d["rows"], d["cols"], d["seed"]
        X = _field(r, c, seed)
        a = B.compress(X)
        if d["op"] == "compress":
            out = B.CMat.empty(r, c)
            ops.append({"op": "compress", "A": X, "out": out})
            meta.append(("compress", X, out))
        elif d["op"] in ("add", "sub"):
            b = B.compress(_field(r, c, seed + 1))
            out = B.CMat.empty(r, c)
            ops.append({"op": d["op"], "a": a, "b": b, "out": out})
            meta.append((d["op"], a, b, out))
        elif d["op"] == "scale":
            out = B.CMat.empty(r, c)
            ops.append({"op": "scale", "a": a, "c": d["c"], "out": out})
            meta.append(("scale", a, d["c"], out))
        elif d["op"] == "dot":
            b = B.compress(_field(r, c, seed + 1))
            res = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            ops.append({"op": "dot", "a": a, "b": b, "result": res})
            meta.append(("dot", a, b, res))
        elif d["op"] == "matmul":
            Bd = torch.randn(c, d["m"], dtype=torch.float64, device="cuda",
                             generator=torch.Generator("cuda").manual_seed(seed))
            C = torch.full((r, d["m"]), np.nan, dtype=torch.float64, device="cuda")
            ops.append({"op": "matmul", "a": a, "B": Bd, "C": C})
            meta.append(("matmul", a, Bd, C))
        if with_decompress and i % 7 == 0:
            D = torch.full((r, c), np.nan, dtype=torch.float64, device="cuda")
            ops.append({"op": "decompress", "a": a, "C": D})
            meta.append(("decompress", a, D))
    return ops, meta


def same_cmat(x, y):
    for u, v in zip(x.to_host(), y.to_host()):
        u, v = np.asarray(u), np.asarray(v)
        if u.dtype == np.float64:
            assert np.array_equal(u.view(np.uint64), v.view(np.uint64))
        else:
            assert np.array_equal(u, v)


def check_against_single_ops(B, meta):
    for m in meta:
        kind = m[0]
        if kind == "compress":
            same_cmat(m[2], B.compress(m[1]))
        elif kind == "add":
            same_cmat(m[3], B.add(m[1], m[2]))
        elif kind == "sub":
            same_cmat(m[3], B.sub(m[1], m[2]))
        elif kind == "scale":
            same_cmat(m[3], B.scale(m[1], m[2]))
        elif kind == "dot":
            alone = float(B.dot(m[1], m[2]).item())
            absum = float((B.decompress(m[1]).abs() * B.decompress(m[2]).abs()).sum())
            assert abs(float(m[3].item()) - alone) <= 2e-12 * absum
        elif kind == "decompress":
            alone = B.decompress(m[1])
            scale = alone.abs().max().item() + 1.0
            assert torch.all((m[2] - alone).abs() <= 1e-12 * scale)
        elif kind == "matmul":
            alone = B.matmul(m[1], m[2], mode="fp64")
            bound = B.decompress(m[1]).abs() @ m[2].abs()
            assert torch.all((m[3] - alone).abs() <= 2e-12 * bound + 1e-300)


def test_small_mixed_batch_equals_single_ops(B):
    specs = W.batch_ops(count=40, seed=5, lo=8, hi=256)
    ops, meta = make_batch(B, specs)
    plan = B.Batch(ops)
    plan.run()
    torch.cuda.synchronize()
    assert B.device_status() == 0
    check_against_single_ops(B, meta)
    info = plan.info()
    assert info["ops"] == len(ops) and info["items"] > 0
    # a replay of the graph gives the same results
    first = [m[3].clone() for m in meta if m[0] in ("dot", "matmul")]
    plan.run()
    torch.cuda.synchronize()
    again = [m[3] for m in meta if m[0] in ("dot", "matmul")]
    for x, y in zip(first, again):
        assert torch.equal(x, y)
    plan.free()


def test_small_batch_against_oracle(B):
    specs = [{"op": "compress", "rows": 64, "cols": 136, "seed": 3},
             {"op": "add", "rows": 72, "cols": 64, "seed": 4},
             {"op": "dot", "rows": 128, "cols": 256, "seed": 5},
             {"op": "matmul", "rows": 64, "cols": 96, "m": 40, "seed": 6},
             {"op": "scale", "rows": 8, "cols": 8, "seed": 7, "c": -2.5}]
    ops, meta = make_batch(B, specs, with_decompress=False)
    plan = B.Batch(ops, blocks_per_item=16)
    plan.run()
    torch.cuda.synchronize()
    oc = O.compress(meta[0][1].cpu().numpy())
    f, s, phi, code = meta[0][2].to_host()
    assert np.array_equal(code, oc.code) and np.array_equal(phi, oc.phi) and np.array_equal(s, oc.s)
    X, Y = _field(72, 64, 4).cpu().numpy(), _field(72, 64, 5).cpu().numpy()
    oadd = O.add(O.compress(X), O.compress(Y))
    assert np.array_equal(meta[1][3].code.cpu().numpy(), oadd.code)
    X, Y = _field(128, 256, 5).cpu().numpy(), _field(128, 256, 6).cpu().numpy()
    ref, absref = O.dot(O.compress(X), O.compress(Y))
    assert abs(float(meta[2][3].item()) - ref) <= 1e-12 * absref
    A6 = O.compress(_field(64, 96, 6).cpu().numpy())
    Bd = meta[3][2].cpu().numpy()
    Cref = O.matmul(A6, Bd)
    bound = np.abs(O.decompress(A6)) @ np.abs(Bd)
    assert np.all(np.abs(meta[3][3].cpu().numpy() - Cref) <= 1e-12 * bound)
    plan.free()


def test_batch_compress_at_certification_boundaries(B, boundary_blocks):
    """The batch kernel's compressor (certified fp32 decisions, exact
    binary64 fix-up inside the item) on the blocks closest to a phi or code
    rounding boundary, against the oracle bit for bit."""
    blk = boundary_blocks[0]
    X = np.ascontiguousarray(blk.transpose(1, 0, 2).reshape(8, -1))
    Y = np.concatenate([X, X[:, ::-1]], axis=0)
    ops, outs = [], []
    for M in (X, Y):
        out = B.CMat.empty(*M.shape)
        ops.append({"op": "compress", "A": torch.from_numpy(M).cuda(), "out": out})
        outs.append((M, out))
    plan = B.Batch(ops, blocks_per_item=16)
    plan.run()
    torch.cuda.synchronize()
    for M, out in outs:
        oc = O.compress(M)
        f, s, phi, code = out.to_host()
        assert np.array_equal(phi, oc.phi) and np.array_equal(code, oc.code)
        assert np.array_equal(s.view(np.uint64), oc.s.view(np.uint64))
        assert np.array_equal(f.view(np.uint64), oc.f.view(np.uint64))
    plan.free()


def test_autotuned_batch_and_aliasing_rule(B):
    specs = W.batch_ops(count=30, seed=8, lo=64, hi=512)
    ops, meta = make_batch(B, specs)
    plan = B.Batch(ops, autotune=True)
    info = plan.info()
    assert info["tuned_ms"] > 0 and info["blocks_per_item"] in (64, 128, 256, 512, 1024)
    plan.run()
    torch.cuda.synchronize()
    check_against_single_ops(B, meta)
    plan.free()
    a = B.compress(_field(64, 64, 1))
    with pytest.raises(B.BlazError) as e:
        B.Batch([{"op": "scale", "a": a, "c": 2.0, "out": a}], autotune=True)
    assert e.value.status == -9


def test_empty_and_degenerate_batches(B):
    plan = B.Batch([])
    plan.run()
    plan.free()
    a = B.compress(torch.zeros((0, 16), dtype=torch.float64, device="cuda"))
    res = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    C = torch.full((16, 8), np.nan, dtype=torch.float64, device="cuda")
    z = B.compress(torch.zeros((16, 0), dtype=torch.float64, device="cuda"))
    plan = B.Batch([{"op": "dot", "a": a, "b": a, "result": res},
                    {"op": "matmul", "a": z, "B": torch.zeros((0, 8), dtype=torch.float64, device="cuda"), "C": C}])
    plan.run()
    torch.cuda.synchronize()
    assert float(res.item()) == 0.0
    assert float(C.abs().max()) == 0.0
    plan.free()


def test_full_batch_workload_sampled(B):
    """2000 ops, sides log-uniform over multiples of 8 in [64, 2048], mix
    40/30/15/10/5 %: every 50th op is checked against the op run alone and
    every 200th compress/add against the oracle."""
    specs = W.batch_ops(count=2000, seed=11)
    ops, meta = make_batch(B, specs, with_decompress=False)
    plan = B.Batch(ops, autotune=True)
    plan.run()
    torch.cuda.synchronize()
    assert B.device_status() == 0
    check_against_single_ops(B, meta[::50])
    for k, m in enumerate(meta):
        if k % 200 == 0 and m[0] == "compress":
            oc = O.compress(m[1].cpu().numpy())
            assert np.array_equal(m[2].code.cpu().numpy(), oc.code)
            assert np.array_equal(m[2].s.cpu().numpy().view(np.uint64), oc.s.view(np.uint64))
    plan.free()
