import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libblaz")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def split_bf16_tol(k):
    """(|A_hat||B|)_ij multiplier of the split-bf16 product: fp32 accumulation
    over the 6k slice products plus the three-slice representation error
    (about 2^-24 of each operand)."""
    return (6 * k + 8) * 2.0 ** -24


# Componentwise error limit of the split-bf16 product for inner dimensions
# k >= 1024, beside the worst-case bound above.  With random-signed operands
# the fp32 accumulation error grows like sqrt(k) 2^-24, not k 2^-24 (measured
# about 4e-6 at k = 4096), while leaving out the slice products of the second
# level (A1 B2 + A2 B1, about 2^-9 of each term) costs about 3e-4 at k = 1024
# (test_split_bf16_model.py emulates both).
SPLIT_BF16_LARGE_K_TOL = 2e-5


def load_golden(name):
    """Parse a tests/golden/*.txt fixture into {section: [rows of tokens]}."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line[1:line.index("]")]
                out[cur] = []
                continue
            out[cur].append(line.split())
    return out


@pytest.fixture(scope="session")
def boundary_blocks():
    """Blocks where the decisions of Eqs. eqphi / eqquant are closest to a
    rounding boundary: 127/m nearest an integer (phi) and X phi nearest a
    nonzero integer (the truncated code), picked by the oracle out of a
    seeded pool of 131072 smooth and rough blocks.  These are the blocks a
    compressor with any approximate shortcut is most likely to get wrong."""
    import numpy as np

    import oracle as O
    import workloads as W

    parts = []
    for seed in range(31, 39):
        parts += [W.random_block_matrix(256, 1024, seed, "smooth"),
                  W.random_block_matrix(256, 1024, seed + 100, "noise"),
                  W.bump_field(1024, seed, rows=256),
                  W.random_block_matrix(256, 1024, seed + 200, "smooth") ** 3]
    pool = np.concatenate(parts, axis=0)
    blocks = pool.reshape(pool.shape[0] // 8, 8, pool.shape[1] // 8, 8).transpose(0, 2, 1, 3).reshape(-1, 8, 8)
    kp = O.kept_positions()
    kr, kc = kp[:, 0], kp[:, 1]
    dphi, dcode = np.full(len(blocks), np.inf), np.full(len(blocks), np.inf)
    for n, blk in enumerate(blocks):
        st = O.block_stages(blk)
        if st["K"] == 0 or not np.isfinite(st["m"]) or st["m"] == 0.0:
            continue
        q = 127.0 / st["m"]
        if 1.0 <= q < 255.0:
            dphi[n] = abs(q - round(q)) / q
        v = np.abs(st["dct"][kr, kc] * st["phi"])
        v = v[(v >= 0.5) & (v < 127.5)]
        if v.size:
            dcode[n] = np.min(np.abs(v - np.round(v)))
    pick = np.unique(np.concatenate([np.argsort(dphi)[:192], np.argsort(dcode)[:192]]))
    return blocks[pick], dphi[pick], dcode[pick]
