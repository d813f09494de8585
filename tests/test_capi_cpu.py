"""CPU checks of the C ABI boundary (no GPU compute calls).

The library builds for sm_103a and loads; it exports every function that
include/qed.h declares; the ctypes mirrors of the header's structs have the
same sizes and field offsets as the C compiler gives them; argument
validation rejects invalid descriptors before touching the device.
"""
import ctypes
import math
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qed.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1412_6426_gb300 import build, qed
    build.build()
    return qed.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(qed_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    from paper_1412_6426_gb300 import qed
    names = declared_functions()
    assert len(names) >= 9
    assert sorted(qed.EXPORTS) == names
    nm = subprocess.run(["nm", "-D", "--defined-only", qed.LIB_PATH], capture_output=True, text=True,
                        check=True).stdout
    exported = set(re.findall(r"\bT (qed_\w+)", nm))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_library_targets_sm103a_only():
    from paper_1412_6426_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_error_strings(lib):
    from paper_1412_6426_gb300 import qed
    assert qed.qed_error_string(0) == "ok"
    assert "capacity" in qed.qed_error_string(qed.QED_ERR_CAPACITY)
    assert qed.qed_error_string(99) == "unknown status"


LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "qed.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("qed_grid_desc %zu\nqed_species_desc %zu\nqed_params %zu\nqed_fields %zu\nqed_diag %zu\n"
         "qed_tuning %zu\n",
         sizeof(qed_grid_desc), sizeof(qed_species_desc), sizeof(qed_params), sizeof(qed_fields),
         sizeof(qed_diag), sizeof(qed_tuning));
  P(qed_grid_desc, d); P(qed_grid_desc, field_mode); P(qed_grid_desc, fp);
  P(qed_params, seed); P(qed_params, kappa); P(qed_params, pending_capacity);
  P(qed_params, ens_bits); P(qed_params, thin_interval); P(qed_params, thin_limit);
  P(qed_params, emit_fg); P(qed_params, pair_fg); P(qed_params, emit_ng); P(qed_params, pair_ng);
  P(qed_params, generator); P(qed_params, reserved_gen); P(qed_params, schwinger_on);
  P(qed_params, schwinger_weight); P(qed_diag, schwinger_pairs); P(qed_diag, schwinger_gt1);
  P(qed_diag, photons_created); P(qed_diag, pairs_created); P(qed_diag, thinned);
  P(qed_diag, kernel_launches);
  P(qed_tuning, work_chunk); P(qed_tuning, sort_massive); P(qed_tuning, concurrent);
  P(qed_tuning, deposit_halo); P(qed_tuning, refill_lanes);
  P(qed_diag, block_steps); P(qed_diag, tile_deposits);
  P(qed_diag, particle_steps); P(qed_diag, species_steps); P(qed_diag, emissions);
  P(qed_diag, time); P(qed_diag, status); P(qed_diag, spectrum);
  P(qed_species_desc, charge); P(qed_fields, J);
  return 0;
}
"""


def test_struct_layouts_match_header(tmp_path):
    from paper_1412_6426_gb300 import qed
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in lines if l.strip())
    m = {"qed_grid_desc": qed.QedGridDesc, "qed_species_desc": qed.QedSpeciesDesc,
         "qed_params": qed.QedParams, "qed_fields": qed.QedFields, "qed_diag": qed.QedDiag,
         "qed_tuning": qed.QedTuning}
    for k, v in got.items():
        if "." in k:
            t, f = k.split(".")
            assert getattr(m[t], f).offset == int(v), k
        else:
            assert ctypes.sizeof(m[k]) == int(v), k


def test_header_constants_match_binding():
    from paper_1412_6426_gb300 import qed, workloads
    text = open(HEADER).read()
    consts = dict(re.findall(r"#define (QED_\w+)\s+(\d+)", text))
    assert int(consts["QED_ENS_STRIDE"]) == qed.QED_ENS_STRIDE == workloads.ENS_STRIDE
    assert int(consts["QED_MAX_ENS_BITS"]) == qed.QED_MAX_ENS_BITS
    assert int(consts["QED_ABI_VERSION"]) == 3
    modes = dict(re.findall(r"(QED_FIELD_\w+) = (\d+)", text))
    assert int(modes["QED_FIELD_ENSEMBLE"]) == qed.QED_FIELD_ENSEMBLE == workloads.FIELD_ENSEMBLE
    assert int(modes["QED_FIELD_STANDING_WAVE"]) == qed.QED_FIELD_STANDING_WAVE == workloads.FIELD_STANDING_WAVE
    stages = re.findall(r"(QED_STAGE_\w+|QED_NSTAGES)\b", text[text.index("typedef enum qed_stage"):])
    order = list(dict.fromkeys(stages))
    assert order[:11] == ["QED_STAGE_BEGIN", "QED_STAGE_CONSTANTS", "QED_STAGE_PHOTONS", "QED_STAGE_BLOCKS",
                          "QED_STAGE_DEPOSIT", "QED_STAGE_MASSIVE", "QED_STAGE_PRODUCTS", "QED_STAGE_SCHWINGER",
                          "QED_STAGE_FIELD", "QED_STAGE_END", "QED_NSTAGES"]
    for k, name in enumerate(order[:11]):
        assert getattr(qed, name) == k


def _descs():
    from paper_1412_6426_gb300 import qed
    g = qed.QedGridDesc()
    g.n[:] = [4, 4, 4]
    g.periodic[:] = [1, 1, 1]
    g.d[:] = [1.0, 1.0, 1.0]
    g.field_mode = qed.QED_FIELD_UNIFORM
    s = qed.QedSpeciesDesc()
    s.capacity[:] = [10, 10, 10, 0]
    s.charge[:] = [-1, 1, 0, 1]
    s.mass[:] = [1, 1, 0, 1836]
    p = qed.QedParams()
    p.precision = 64
    p.nsub_max = 10
    p.kappa = 0.1
    return g, s, p


@pytest.mark.parametrize("bad", ["precision", "cells", "grid_open", "kappa", "nbins", "mass", "tables",
                                 "ens_bits", "thin_limit", "fg_nan", "ng", "mode", "generator",
                                 "generator_factor", "schwinger_weight", "schwinger_ensemble"])
def test_argument_validation(lib, bad):
    from paper_1412_6426_gb300 import qed
    g, s, p = _descs()
    tables = None
    if bad == "precision":
        p.precision = 16
    elif bad == "cells":
        g.n[1] = 0
    elif bad == "grid_open":
        g.field_mode = qed.QED_FIELD_GRID
        g.periodic[2] = 0
    elif bad == "kappa":
        p.kappa = -1.0
    elif bad == "nbins":
        p.nbins = 5000
    elif bad == "mass":
        s.mass[0] = 0.0
    elif bad == "tables":
        tables = b"\0" * 7
    elif bad == "ens_bits":
        p.ens_bits = 17
    elif bad == "thin_limit":
        p.thin_limit[2] = -1
    elif bad == "fg_nan":
        p.emit_fg = float("nan")
    elif bad == "ng":
        p.pair_ng = 65
    elif bad == "mode":
        g.field_mode = 6
    elif bad == "generator":
        p.generator = 3
    elif bad == "generator_factor":
        p.generator = 2
        p.emit_fg = 2.0
    elif bad == "schwinger_weight":
        p.schwinger_on = 1
        p.schwinger_weight = 0.0
    elif bad == "schwinger_ensemble":
        p.schwinger_on = 1
        p.schwinger_weight = 1.0
        g.field_mode = qed.QED_FIELD_ENSEMBLE
    with pytest.raises(qed.QedError) as e:
        qed.qed_init(g, s, p, tables=tables)
    assert e.value.status == qed.QED_ERR_ARG


def test_null_arguments(lib):
    from paper_1412_6426_gb300 import qed
    assert lib.qed_init(None, None, None, None, 0, None, None) == qed.QED_ERR_ARG
    assert lib.qed_step(None, None, 1.0, 1, None) == qed.QED_ERR_ARG
    assert lib.qed_ensembles_set(None, 1, None, None) == qed.QED_ERR_ARG
    assert lib.qed_get_tuning(None, None) == qed.QED_ERR_ARG
    assert lib.qed_set_tuning(None, None) == qed.QED_ERR_ARG
    assert lib.qed_autotune(None, None, 1.0, 1, 10, None, None, None) == qed.QED_ERR_ARG
    assert lib.qed_destroy(None) == qed.QED_OK
    assert lib.qed_diagnostics(None, None, None) == qed.QED_ERR_ARG
    assert lib.qed_selftest_barrier(None, -1, 1, None) == qed.QED_ERR_ARG
    assert lib.qed_profile_stages(None, None, 0) == qed.QED_ERR_ARG
    assert lib.qed_particles_read_static(None, 0, None, None, None, None, 0, None, None) == qed.QED_ERR_ARG


def test_product_path_has_no_oracle_import():
    # the product package never imports the oracle, and fails loudly without its library
    pkg = os.path.join(ROOT, "paper_1412_6426_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            assert "oracle" not in re.sub(r'""".*?"""', "", open(os.path.join(pkg, f)).read(), flags=re.S), f
    code = ("import paper_1412_6426_gb300.qed as q; q.LIB_PATH='/nonexistent.so'; q._lib=None\n"
            "try:\n q.load(q.LIB_PATH)\nexcept RuntimeError: print('raised')\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT).stdout
    assert "raised" in out


def test_oracle_and_library_share_no_code():
    # the oracle includes only the C standard library, the library's sources
    # and header name nothing under oracle/, and the oracle's Python side
    # never loads the CUDA library or its package (only the seeded inputs of
    # workloads.py serve both)
    src = open(os.path.join(ROOT, "oracle", "qed_oracle.c")).read()
    assert set(re.findall(r"#include\s*[<\"]([^>\"]+)[>\"]", src)) <= {"math.h", "stdint.h", "stdlib.h", "string.h"}
    lib_files = [os.path.join(ROOT, "paper_1412_6426_gb300", "csrc", f)
                 for f in os.listdir(os.path.join(ROOT, "paper_1412_6426_gb300", "csrc"))]
    for f in lib_files + [HEADER]:
        text = open(f).read()
        assert "oracle" not in text.lower() and "qed_oracle" not in text, f
        for inc in re.findall(r"#include\s*\"([^\"]+)\"", text):
            assert os.path.exists(os.path.join(os.path.dirname(f), inc)) or inc == "qed.h", (f, inc)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            code = re.sub(r'""".*?"""', "", open(os.path.join(ROOT, "oracle", f)).read(), flags=re.S)
            for mod in re.findall(r"^\s*import\s+([\w.]+)", code, re.M):
                assert not mod.startswith("paper_1412_6426_gb300") or mod == "paper_1412_6426_gb300.workloads", (f, mod)
            for mod, names in re.findall(r"^\s*from\s+([\w.]+)\s+import\s+([\w, ]+)", code, re.M):
                if mod == "paper_1412_6426_gb300":
                    assert {n.strip() for n in names.split(",")} <= {"workloads"}, (f, names)
                else:
                    assert not mod.startswith("paper_1412_6426_gb300.") or mod == "paper_1412_6426_gb300.workloads", (f, mod)
            assert "libqed_gb300" not in code and "qed.load" not in code, f
    # no table of numbers typed on both sides: the long literals they share
    # are the published CODATA constants alone
    num = re.compile(r"(?<![\w.])(\d+\.\d{6,}(?:e[+-]?\d+)?)")
    oracle_lits = set(num.findall(src))
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            oracle_lits |= set(num.findall(open(os.path.join(ROOT, "oracle", f)).read()))
    pkg = os.path.join(ROOT, "paper_1412_6426_gb300")
    lib_lits = set()
    for f in lib_files + [HEADER] + [os.path.join(pkg, g) for g in os.listdir(pkg) if g.endswith(".py")]:
        lib_lits |= set(num.findall(open(f).read()))
    assert oracle_lits & lib_lits <= {"7.2973525693e-3", "1836.15267343"}, oracle_lits & lib_lits


def test_device_gauss_legendre_constants():
    # the 8-point Gauss-Legendre nodes and weights the FP64 standard generator
    # integrates with (written into the device header) against the roots of
    # P_8 and their weights 2 / ((1 - x^2) P_8'(x)^2), found to 30 digits
    mpmath = pytest.importorskip("mpmath")
    text = open(os.path.join(ROOT, "paper_1412_6426_gb300", "csrc", "qed_device.cuh")).read()
    body = text[text.index("double std_gl8("):]
    x = [float(v) for v in re.search(r"const double x\[4\] = \{([^}]*)\}", body).group(1).split(",")]
    w = [float(v) for v in re.search(r"const double w\[4\] = \{([^}]*)\}", body).group(1).split(",")]
    mpmath.mp.dps = 30
    P8 = lambda t: mpmath.legendre(8, t)
    for xi, wi in zip(x, w):
        r = mpmath.findroot(P8, xi)
        wt = 2 / ((1 - r ** 2) * mpmath.diff(P8, r) ** 2)
        assert xi == float(r) and wi == float(wt)


def test_device_constants():
    # the literal constants of the device header against their definitions:
    # the CODATA 2018 fine-structure constant, sqrt(3)/(2 pi) correctly
    # rounded, pi, and the
    # standard generator's table rows, ln chi from ln 1e-6 in 4096 steps to
    # ln 1e4
    text = open(os.path.join(ROOT, "paper_1412_6426_gb300", "csrc", "qed_device.cuh")).read()

    def const(name):
        m = re.search(r"constexpr (?:double|int) (?:\w+ = [^,;]+, )*" + name + r" = ([^,;]+)[,;]", text)
        return eval(m.group(1), {"__builtins__": {}})      # a literal or a literal quotient

    assert const("kAlpha") == 7.2973525693e-3
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    assert const("kSqrt3Over2Pi") == float(mpmath.sqrt(3) / (2 * mpmath.pi))   # correctly rounded
    assert const("kPi") == math.pi and const("kTwoPi") == 2 * math.pi
    assert const("kStdLnChiLo") == math.log(1e-6)
    assert abs(const("kStdDLn") * 4096 - math.log(1e10)) < 1e-14
    assert const("kStdRows") == 4097 and const("kStdCols") == 1025


def test_fast_division_is_exact(tmp_path):
    # the multiply-shift division that splits cell indices and forms the cell
    # sort's keys, for the divisors the meshes give (edges, planes, cell-block
    # counts), checked on the host against integer division for n < 2^31
    from paper_1412_6426_gb300 import build
    exe = str(tmp_path / "fast_div")
    subprocess.run([build.nvcc(), "-O2", "-std=c++17", "-I", build.CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "fast_div_host.cu"), "-o", exe], check=True)
    divisors = [1, 2, 3, 7, 8, 12, 16, 64, 100, 255, 256, 257, 511, 512, 513, 1000, 4096, 65536, 65537,
                262144, 2 ** 20 - 1, 2 ** 24 + 3, 1_000_003, 2 ** 30, 2 ** 31 - 1]
    out = subprocess.run([exe, *map(str, divisors)], capture_output=True, text=True, check=True).stdout.split()
    misses, tried = int(out[0]), int(out[1])
    assert tried > len(divisors) * (1 << 20) and misses == 0, (misses, tried)
