"""Known-answer pin of Philox4x32-10 (Salmon et al., SC'11), the generator
behind every r1, r2 of the event generators (Sec. IV.F-G, V.A) and every
product id.

The oracle's generator is compared word for word with two implementations
written independently of this project: PyTorch's ATen Philox engine (a C++
header, compiled here into a small program; CPU test) and cuRAND's
curand_Philox4x32_10 (GPU test, which also runs the library's own device
generator on the same inputs).  The inputs are 10^4 seeded random (counter,
key) pairs plus the corner cases of all-zero and all-one words.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as o

HERE = os.path.dirname(os.path.abspath(__file__))


def cases(n=10_000, seed=20141219):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 2 ** 32, size=(n, 6), dtype=np.uint64)
    edge = np.array([[0] * 6, [2 ** 32 - 1] * 6, [0, 0, 0, 0, 2 ** 32 - 1, 2 ** 32 - 1],
                     [2 ** 32 - 1] * 4 + [0, 0]], dtype=np.uint64)
    return np.concatenate([edge, a])


def oracle_words(c):
    return np.array([o.philox([int(v) for v in row[:4]], [int(v) for v in row[4:]]) for row in c],
                    dtype=np.uint64)


def run_program(exe, c):
    text = "\n".join(" ".join(str(int(v)) for v in row) for row in c) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    return np.array([[int(v) for v in line.split()] for line in out.strip().splitlines()], dtype=np.uint64)


def test_oracle_philox_matches_aten(tmp_path):
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    cxx = shutil.which("g++")
    if not os.path.exists(hdr) or cxx is None:
        pytest.skip("ATen Philox header or g++ not available")
    exe = str(tmp_path / "philox_aten")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", inc, os.path.join(HERE, "native", "philox_aten.cpp"),
                    "-o", exe], check=True)
    c = cases()
    ref = run_program(exe, c)
    assert ref.shape == (len(c), 4)
    assert np.array_equal(oracle_words(c), ref)


@pytest.mark.gpu
def test_device_philox_matches_curand_and_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1412_6426_gb300 import build
    exe = str(tmp_path / "philox_curand")
    subprocess.run([build.nvcc(), *build.ARCH, "-O2", "-std=c++17", "-I", build.CSRC,
                    os.path.join(HERE, "native", "philox_curand.cu"), "-o", exe], check=True)
    c = cases()
    out = run_program(exe, c)
    assert out.shape == (len(c), 8)
    lib, ref = out[:, :4], out[:, 4:]
    assert np.array_equal(lib, ref)                  # the library's generator is cuRAND's
    assert np.array_equal(lib, oracle_words(c))      # and the oracle's
