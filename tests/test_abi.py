"""The C-ABI library loads on the CPU host, exports every entry point of
include/dbm.h, and its host-side validation (dbm_init, no GPU involved)
accepts and rejects parameters as documented."""
import os
import re

import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def D():
    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm

    B.build()
    dbm.load()
    return dbm


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "dbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dbm_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dbm_init", "dbm_step", "dbm_moments", "dbm_nonequilibrium", "dbm_set_state",
                     "dbm_conservation", "dbm_status", "dbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(D):
    import ctypes

    lib = ctypes.CDLL(D.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_declared_functions()) <= set(D.EXPORTS) | set()


def _params(D, **over):
    pb = W.random_smooth(16, 8, 2)
    for k, v in over.items():
        setattr(pb, k, v)
    return D.params_from_problem(pb, "fp32")


def test_init_accepts_a_valid_problem(D):
    h = D.dbm_init(_params(D))
    lay = D.dbm_get_layout(h)
    assert lay.pitch % 32 == 0 and lay.pitch >= 16 + 4 + 2
    assert lay.rows == 8 + 4 and lay.gx == 4 and lay.gy == 2
    assert D.dbm_state_bytes(h) == 2 * 16 * lay.plane * 4
    assert D.dbm_scratch_bytes(h) >= 256
    assert D.dbm_steps_taken(h) == 0
    D.dbm_destroy(h)


def test_layout_per_precision(D):
    pb = W.random_smooth(100, 7, 3)
    for prec, eb in (("fp64", 8), ("fp32", 4)):
        h = D.dbm_init(D.params_from_problem(pb, prec))
        lay = D.dbm_get_layout(h)
        assert lay.elem_bytes == eb
        assert lay.bytes == 3 * 16 * lay.plane * eb
        D.dbm_destroy(h)


@pytest.mark.parametrize("case,code", [
    (dict(nx=0), -1),
    (dict(dt=-1.0), -1),
    (dict(dt=1e-3), -7),           # CFL
    (dict(bc_x=5), -1),
])
def test_init_rejects(D, case, code):
    with pytest.raises(D.DbmError) as e:
        D.dbm_init(_params(D, **case))
    assert e.value.code == code
    assert len(str(e.value)) > 20


def test_init_rejects_bad_species(D):
    pb = W.random_smooth(8, 8, 2)
    pb.species[1].eta = (0.0, 0.0, 0.0, 0.0)  # singular moment matrix
    with pytest.raises(D.DbmError) as e:
        D.dbm_init(D.params_from_problem(pb))
    assert e.value.code == -2
    pb = W.random_smooth(8, 8, 2)
    pb.species[0].tau = 0.0
    with pytest.raises(D.DbmError):
        D.dbm_init(D.params_from_problem(pb))
    pb = W.random_smooth(8, 8, 2)
    pb.species[0].tau = 4e-6  # dt >= 2 tau
    with pytest.raises(D.DbmError) as e:
        D.dbm_init(D.params_from_problem(pb))
    assert e.value.code == -7
    pb = W.random_smooth(8, 8, 9 - 1)
    pb.species.append(pb.species[0])  # 9 species
    with pytest.raises(ValueError):
        D.params_from_problem(pb)


def test_init_rejects_mass_creating_reaction(D):
    pb = W.random_smooth(8, 8, 3, reactive=True)
    h = D.dbm_init(D.params_from_problem(pb))
    D.dbm_destroy(h)
    pb.species[2].a = 1.5  # sum a m != 0
    with pytest.raises(D.DbmError) as e:
        D.dbm_init(D.params_from_problem(pb))
    assert "conserve mass" in str(e.value)
    pb = W.random_smooth(8, 8, 3, reactive=True)
    pb.fuel = 7
    with pytest.raises(D.DbmError):
        D.dbm_init(D.params_from_problem(pb))


def test_condition_check_is_unit_independent(D):
    """The same velocity set in other velocity units (v and eta scaled by
    300) is accepted: the check uses the row-equilibrated matrix."""
    pb = W.random_smooth(8, 8, 1)
    sp = pb.species[0]
    sp.v = tuple(300 * x for x in sp.v)
    sp.eta = tuple(300 * x for x in sp.eta)
    pb.dt = 1e-8
    pb.species[0].tau = 2e-8
    h = D.dbm_init(D.params_from_problem(pb))
    D.dbm_destroy(h)


def test_calls_without_buffers_fail_cleanly(D):
    h = D.dbm_init(_params(D))
    with pytest.raises(D.DbmError) as e:
        D.dbm_step(h, 1, 0)
    assert e.value.code == -3
    with pytest.raises(D.DbmError):
        D.dbm_bind(h, 0, 0, 0)
    D.dbm_destroy(h)
    D.dbm_destroy(None)


def test_equilibrium_matrix_is_correctly_rounded(D):
    """The library's M^-1 (host FP64, its own LU and refinement) equals the
    exact rational inverse of M rounded to double in every nonzero entry,
    like the oracle's: the two sides then share the same equilibrium
    operator without sharing code."""
    from tests.test_oracle_pins import _exact_inverse

    pb = W.random_smooth(8, 8, 3)
    h = D.dbm_init(D.params_from_problem(pb))
    try:
        for s, sp in enumerate(pb.species):
            Mi = D.dbm_equilibrium_matrix(h, s)
            # M rebuilt here from the velocity set, row k = moment monomial k
            M = _moment_matrix_from_velocities(sp)
            E = _exact_inverse(M)
            nz = E != 0
            assert np.array_equal(Mi[nz], E[nz])
            assert np.max(np.abs(Mi[~nz])) <= 1e-30 * np.max(np.abs(E))
    finally:
        D.dbm_destroy(h)


def _moment_matrix_from_velocities(sp):
    dirs = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    M = np.zeros((16, 16))
    for i in range(16):
        r = i // 4
        dx, dy = dirs[(4 if r % 2 else 0) + i % 4]
        x, y = dx * sp.v[r], dy * sp.v[r]
        q = x * x + y * y + sp.eta[r] * sp.eta[r]
        M[:, i] = [1.0, x, y, q, x * x, x * y, y * y, q * x, q * y, x * x * x, x * x * y, x * y * y,
                   y * y * y, q * x * x, q * x * y, q * y * y]
    return M


def test_step_kernel_choices(D):
    """Unknown kernels, the two-cell steps outside FP32 with two or more
    species, the one-cell TMA step beyond four species, the species-staged
    step with an arithmetic option (or the two-cell step for three species
    with one) and a TMA kernel for BF16DEV are refused at init; the tile is
    known only once buffers are bound."""
    pb1, pb2, pb3 = W.random_smooth(8, 8, 1), W.random_smooth(8, 8, 2), W.random_smooth(8, 8, 3)
    pb5 = W.random_smooth(8, 8, 5)
    for pb, prec, kern, opts in ((pb2, "fp32", 6, {}), (pb2, "fp32", -1, {}), (pb1, "fp32", "tma_pair", {}),
                                 (pb1, "fp32", "tma_staged", {}), (pb5, "fp32", "tma_cell", {}),
                                 (pb2, "fp32", "tma_staged", {"rounding": "stochastic"}),
                                 (pb3, "fp32", "tma_pair", {"thermo": "fp64"}),
                                 (pb2, "fp64", "tma_pair", {}), (pb3, "fp64", "tma_staged", {}),
                                 (pb2, "bf16dev", "tma_cell", {})):
        with pytest.raises(D.DbmError) as e:
            D.dbm_init(D.params_from_problem(pb, prec, kern, **opts))
        assert e.value.code == -1, (prec, kern, opts)
    for pb, kern in ((pb3, "tma_pair"), (pb2, "tma_staged"), (pb5, "tma_staged"), (pb2, "tma_pair")):
        D.dbm_destroy(D.dbm_init(D.params_from_problem(pb, "fp32", kern)))
    h = D.dbm_init(D.params_from_problem(pb2, "fp32", "tma_pair"))
    with pytest.raises(D.DbmError) as e:
        D.dbm_step_tile(h)
    assert e.value.code == -3
    D.dbm_destroy(h)
    with pytest.raises(ValueError):
        D.params_from_problem(pb2, "fp32", "tma_quad")
    with pytest.raises(ValueError):
        D.params_from_problem(pb2, "fp16")


def test_bf16dev_scope(D):
    """BF16-deviation storage: up to 4 species, no reaction, no force."""
    pb = W.random_smooth(8, 8, 2)
    h = D.dbm_init(D.params_from_problem(pb, "bf16dev"))
    lay = D.dbm_get_layout(h)
    assert lay.elem_bytes == 2 and lay.moments_offset % 256 == 0
    assert lay.bytes == lay.moments_offset + (2 + 3) * lay.plane * 4
    D.dbm_destroy(h)
    for bad in (W.random_smooth(8, 8, 3, reactive=True), W.random_smooth(8, 8, 2, force=True),
                W.random_smooth(8, 8, 5)):
        with pytest.raises(D.DbmError) as e:
            D.dbm_init(D.params_from_problem(bad, "bf16dev"))
        assert "BF16DEV" in str(e.value)


def test_struct_layout_matches_the_header(D, tmp_path):
    """The binding's ctypes records have the size and field offsets that a
    C compiler gives the structs of include/dbm.h."""
    import ctypes
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    fields = [name for name, _ in D.dbm_params._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dbm.h"', "int main(void) {",
             '  printf("params %zu\\n", sizeof(dbm_params));',
             '  printf("layout %zu\\n", sizeof(dbm_layout));',
             '  printf("species %zu\\n", sizeof(dbm_species));']
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof(dbm_params, {f}));')
    lines.append("  return 0; }")
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    assert int(out["params"]) == ctypes.sizeof(D.dbm_params)
    assert int(out["layout"]) == ctypes.sizeof(D.dbm_layout)
    assert int(out["species"]) == ctypes.sizeof(D.dbm_species)
    for f in fields:
        assert int(out[f]) == getattr(D.dbm_params, f).offset, f


def test_arithmetic_options_scope(D):
    """The thermo and rounding options exist for the TMA-staged FP32 step
    with up to 4 species; elsewhere, and for unknown values, init refuses."""
    pb2, pb5 = W.random_smooth(8, 8, 2), W.random_smooth(8, 8, 5)
    ok = D.dbm_init(D.params_from_problem(pb2, "fp32", thermo="fp64", rounding="stochastic"))
    D.dbm_destroy(ok)
    for pb, prec, kern, opts in ((pb2, "fp64", "auto", dict(thermo="fp64")),
                                 (pb2, "bf16dev", "auto", dict(rounding="stochastic")),
                                 (pb5, "fp32", "auto", dict(thermo="fp64")),
                                 (pb2, "fp32", "generic", dict(rounding="stochastic")),
                                 (pb2, "fp32", "auto", dict(thermo=7)),
                                 (pb2, "fp32", "auto", dict(rounding=-1))):
        with pytest.raises(D.DbmError) as e:
            D.dbm_init(D.params_from_problem(pb, prec, kern, **opts))
        assert e.value.code == -1, (prec, kern, opts)
    with pytest.raises(ValueError):
        D.params_from_problem(pb2, "fp32", thermo="fp128")
    with pytest.raises(ValueError):
        D.params_from_problem(pb2, "fp32", rounding="up")
