"""The bounds-checked build (-DDBM_CHECKED), a debugging aid in place of a
memory checker: every index into a shared-memory tile, a state buffer or a
ghost image is compared with the extent of what it addresses; one outside
it raises DBM_HEALTH_BOUNDS (bit 32) and the access is skipped.

Small grids with ragged tiles, one- and two-cell tiles, the species-staged
tile for two to eight species, every boundary pairing, the generic, FP64 and BF16DEV steps and every batched tile shape
run in a child process on the checked library; no case may raise bit 32,
and every final state must equal, bit for bit, the same case run on the
normal library in this process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BOUNDS_BIT = 32

PO, PP, OO, OP = (W.PERIODIC, W.OUTFLOW), (W.PERIODIC, W.PERIODIC), (W.OUTFLOW, W.OUTFLOW), (W.OUTFLOW, W.PERIODIC)
CASES = [  # name, nx, ny, species, precision, kernel, boundaries
    ("cell_33x21", 33, 21, 2, "fp32", "tma_cell", PO),
    ("pair_65x5", 65, 5, 2, "fp32", "tma_pair", OO),
    ("pair_131x10", 131, 10, 2, "fp32", "tma_pair", OP),
    ("one_1x1", 1, 1, 2, "fp32", "auto", PP),
    ("three_2x3", 2, 3, 3, "fp32", "auto", PP),
    ("four_37x13", 37, 13, 4, "fp32", "auto", PO),
    ("single_70x23", 70, 23, 1, "fp32", "auto", OP),
    ("generic_45x9_s5", 45, 9, 5, "fp32", "generic", PO),
    ("staged_45x9_s3", 45, 9, 3, "fp32", "tma_pair", PP),
    ("staged_67x9_s2", 67, 9, 2, "fp32", "tma_staged", OO),
    ("staged_45x9_s5", 45, 9, 5, "fp32", "auto", PO),
    ("staged_130x17_s8", 130, 17, 8, "fp32", "auto", OP),
    ("fp64_21x7", 21, 7, 2, "fp64", "auto", OO),
    ("bf16_33x17", 33, 17, 2, "bf16dev", "auto", PO),
    ("bf16_9x5_s1", 9, 5, 1, "bf16dev", "auto", PP),
]
BATCH_SHAPES = [((32, 10), 1), ((32, 8), 1), ((32, 16), 1), ((32, 7), 1), ((64, 4), 1), ((64, 8), 2), ((32, 16), 2)]


def run_cases(out_dir):
    """Run every case on the library this process loaded; final states go to
    out_dir as .npy files; returns the health bits of each case."""
    from paper_2006_15932_gb300 import dbm as D

    D.load()
    bits = {}
    for name, nx, ny, ns, prec, kern, bc in CASES:
        pb = W.random_smooth(nx, ny, ns, seed=nx + 7 * ny, reactive=(ns == 3 and prec == "fp32"), bc=bc)
        s = D.Solver(pb, prec, step_kernel=kern)
        s.set_state()
        s.step(4)
        bits[name] = s.status()[1]
        np.save(os.path.join(out_dir, name + ".npy"), s.get_f().cpu().numpy())
        s.close()
    stream = torch.cuda.Stream()
    pbs = W.batched_instances(3, seed=5, lo=21, hi=70)
    for tile, cells in BATCH_SHAPES:
        for persistent in (0, 1):
            sols = []
            for q in pbs:
                sols.append(D.Solver(q, "fp32", stream=stream))
                sols[-1].set_state()
            batch = D.Batch(sols, stream=stream, config={"tile": tile, "cells": cells, "persistent": persistent,
                                                         "promote": 1})
            batch.step(3)
            name = f"batch_{tile[0]}x{tile[1]}_{cells}_{persistent}"
            bits[name] = max(s_.status()[1] for s_ in sols)
            np.save(os.path.join(out_dir, name + ".npy"),
                    np.concatenate([s_.get_f().cpu().numpy().ravel() for s_ in sols]))
            batch.close()
            for s_ in sols:
                s_.close()
    return bits


def test_checked_build_finds_no_out_of_range_index(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_15932_gb300 import build as B

    lib = B.build(checked=True)
    B.build()
    checked_dir, plain_dir = tmp_path / "checked", tmp_path / "plain"
    checked_dir.mkdir()
    plain_dir.mkdir()
    code = ("import json, sys; sys.path.insert(0, %r); "
            "from tests.test_gpu_checked import run_cases; print(json.dumps(run_cases(%r)))") % (ROOT, str(checked_dir))
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, DBM_LIB=lib), capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    checked_bits = json.loads(r.stdout.strip().splitlines()[-1])
    assert all(b & BOUNDS_BIT == 0 for b in checked_bits.values()), checked_bits
    assert all(b == 0 for b in checked_bits.values()), checked_bits
    plain_bits = run_cases(str(plain_dir))
    assert all(b == 0 for b in plain_bits.values()), plain_bits
    for name in plain_bits:
        a = np.load(plain_dir / (name + ".npy"))
        b = np.load(checked_dir / (name + ".npy"))
        assert np.array_equal(a, b), name
