"""Thin Python binding of the C ABI in ``include/dbm.h`` (``_build/libdbm.so``).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no
fallback: if the shared library is missing or fails to load, every entry
point raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DBM_LIB selects another build of the library (e.g. the bounds-checked one)
LIB_PATH = os.environ.get("DBM_LIB") or os.path.join(HERE, "_build", "libdbm.so")

Q = 16
MAX_SPECIES = 8
PERIODIC, OUTFLOW = 0, 1
FP64, FP32, BF16DEV = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16dev": BF16DEV}

OK = 0
ERRORS = {
    -1: "DBM_ERR_INVALID",
    -2: "DBM_ERR_SINGULAR",
    -3: "DBM_ERR_UNBOUND",
    -4: "DBM_ERR_CUDA",
    -5: "DBM_ERR_NONFINITE",
    -6: "DBM_ERR_NEGATIVE",
    -7: "DBM_ERR_STABILITY",
    -8: "DBM_ERR_TIMEOUT",
    -9: "DBM_ERR_BOUNDS",
}
KERNELS = {"auto": 0, "generic": 1, "tma": 2, "tma_cell": 3, "tma_pair": 4, "tma_staged": 5}
THERMO = {"floatfloat": 0, "fp64": 1}
ROUNDING = {"nearest": 0, "stochastic": 1}
EXPORTS = [
    "dbm_init", "dbm_init_error", "dbm_equilibrium_matrix", "dbm_get_layout", "dbm_state_bytes", "dbm_scratch_bytes",
    "dbm_bind", "dbm_set_state", "dbm_set_f", "dbm_get_f", "dbm_step", "dbm_moments",
    "dbm_nonequilibrium", "dbm_conservation", "dbm_conservation_noalloc", "dbm_status", "dbm_steps_taken",
    "dbm_step_tile",
    "dbm_last_error", "dbm_destroy", "dbm_batch_table_bytes", "dbm_batch_create", "dbm_batch_tune",
    "dbm_batch_step", "dbm_batch_info", "dbm_batch_get_config", "dbm_batch_set_config", "dbm_batch_last_error",
    "dbm_batch_destroy",
]


class DbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class dbm_species(C.Structure):
    _fields_ = [
        ("m", C.c_double),
        ("I", C.c_double),
        ("tau", C.c_double),
        ("v", C.c_double * 4),
        ("eta", C.c_double * 4),
        ("a_stoich", C.c_double),
    ]


class dbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int),
        ("ny", C.c_int),
        ("nspecies", C.c_int),
        ("dx", C.c_double),
        ("dy", C.c_double),
        ("dt", C.c_double),
        ("bc_x", C.c_int),
        ("bc_y", C.c_int),
        ("fuel", C.c_int),
        ("oxidizer", C.c_int),
        ("k_ov", C.c_double),
        ("Ea_over_R", C.c_double),
        ("Q", C.c_double),
        ("accel", C.c_double * 2),
        ("precision", C.c_int),
        ("step_kernel", C.c_int),
        ("wait_polls", C.c_int),
        ("thermo", C.c_int),
        ("rounding", C.c_int),
        ("sp", dbm_species * MAX_SPECIES),
    ]


class dbm_layout(C.Structure):
    _fields_ = [
        ("pitch", C.c_int),
        ("rows", C.c_int),
        ("gx", C.c_int),
        ("gy", C.c_int),
        ("plane", C.c_longlong),
        ("elem_bytes", C.c_int),
        ("moments_offset", C.c_size_t),
        ("bytes", C.c_size_t),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Load libdbm.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2006_15932_gb300.build.build()")
    L = C.CDLL(path)
    H = C.c_void_p
    vp = C.c_void_p
    L.dbm_init.argtypes = [C.POINTER(dbm_params), C.POINTER(H)]
    L.dbm_init_error.restype = C.c_char_p
    L.dbm_equilibrium_matrix.argtypes = [H, C.c_int, vp]
    L.dbm_get_layout.argtypes = [H, C.POINTER(dbm_layout)]
    L.dbm_state_bytes.argtypes = [H, C.POINTER(C.c_size_t)]
    L.dbm_scratch_bytes.argtypes = [H, C.POINTER(C.c_size_t)]
    L.dbm_bind.argtypes = [H, vp, vp, vp]
    L.dbm_set_state.argtypes = [H, vp, vp, vp, vp, vp]
    L.dbm_set_f.argtypes = [H, vp, vp]
    L.dbm_get_f.argtypes = [H, vp, vp]
    L.dbm_step.argtypes = [H, C.c_int, vp]
    L.dbm_moments.argtypes = [H, vp, vp]
    L.dbm_nonequilibrium.argtypes = [H, vp, vp]
    L.dbm_conservation.argtypes = [H, vp, vp]
    L.dbm_conservation_noalloc.argtypes = [H, vp, vp, vp]
    L.dbm_status.argtypes = [H, vp, C.POINTER(C.c_uint)]
    L.dbm_steps_taken.argtypes = [H]
    L.dbm_steps_taken.restype = C.c_longlong
    L.dbm_step_tile.argtypes = [H] + [C.POINTER(C.c_int)] * 3
    L.dbm_last_error.argtypes = [H]
    L.dbm_last_error.restype = C.c_char_p
    L.dbm_destroy.argtypes = [H]
    L.dbm_destroy.restype = None
    HP = C.POINTER(C.c_void_p)
    L.dbm_batch_table_bytes.argtypes = [HP, C.c_int, C.POINTER(C.c_size_t)]
    L.dbm_batch_create.argtypes = [HP, C.c_int, vp, C.c_size_t, vp, C.POINTER(C.c_void_p)]
    L.dbm_batch_tune.argtypes = [vp, vp, C.c_int]
    L.dbm_batch_step.argtypes = [vp, C.c_int, vp]
    L.dbm_batch_info.argtypes = [vp] + [C.POINTER(C.c_int)] * 4
    L.dbm_batch_get_config.argtypes = [vp] + [C.POINTER(C.c_int)] * 5
    L.dbm_batch_set_config.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp]
    L.dbm_batch_last_error.argtypes = [vp]
    L.dbm_batch_last_error.restype = C.c_char_p
    L.dbm_batch_destroy.argtypes = [vp]
    L.dbm_batch_destroy.restype = None
    for name in EXPORTS:
        getattr(L, name)
    _lib = L
    return L


def make_params(nx, ny, species, *, dx, dy, dt, bc_x=PERIODIC, bc_y=PERIODIC, fuel=0, oxid=1,
                k_ov=0.0, Ea_over_R=0.0, Q=0.0, accel=(0.0, 0.0), precision=FP64,
                step_kernel="auto", wait_polls=0, thermo="floatfloat", rounding="nearest") -> dbm_params:
    """Fill a dbm_params record; ``species`` items need m, I, tau, v, eta, a."""
    if len(species) > MAX_SPECIES:
        raise ValueError(f"at most {MAX_SPECIES} species")
    p = dbm_params()
    p.nx, p.ny, p.nspecies = int(nx), int(ny), len(species)
    p.dx, p.dy, p.dt = float(dx), float(dy), float(dt)
    p.bc_x, p.bc_y = int(bc_x), int(bc_y)
    p.fuel, p.oxidizer = int(fuel), int(oxid)
    p.k_ov, p.Ea_over_R, p.Q = float(k_ov), float(Ea_over_R), float(Q)
    p.accel[0], p.accel[1] = float(accel[0]), float(accel[1])
    if isinstance(precision, str) and precision not in PRECISIONS:
        raise ValueError(f"precision {precision!r}: one of {sorted(PRECISIONS)}")
    if isinstance(step_kernel, str) and step_kernel not in KERNELS:
        raise ValueError(f"step_kernel {step_kernel!r}: one of {sorted(KERNELS)}")
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.step_kernel = KERNELS[step_kernel] if isinstance(step_kernel, str) else int(step_kernel)
    p.wait_polls = int(wait_polls)
    for name, val, table in (("thermo", thermo, THERMO), ("rounding", rounding, ROUNDING)):
        if isinstance(val, str) and val not in table:
            raise ValueError(f"{name} {val!r}: one of {sorted(table)}")
        setattr(p, name, table[val] if isinstance(val, str) else int(val))
    for s, sp in enumerate(species):
        c = p.sp[s]
        c.m, c.I, c.tau, c.a_stoich = float(sp.m), float(sp.I), float(sp.tau), float(sp.a)
        for r in range(4):
            c.v[r] = float(sp.v[r])
            c.eta[r] = float(sp.eta[r])
    return p


def params_from_problem(pb, precision=FP64, step_kernel="auto", **opts) -> dbm_params:
    return make_params(pb.nx, pb.ny, pb.species, dx=pb.dx, dy=pb.dy, dt=pb.dt, bc_x=pb.bc_x,
                       bc_y=pb.bc_y, fuel=pb.fuel, oxid=pb.oxid, k_ov=pb.k_ov,
                       Ea_over_R=pb.Ea_over_R, Q=pb.Q, accel=pb.accel, precision=precision,
                       step_kernel=step_kernel, **opts)


# ---------------------------------------------------------------------------
# the C entry points, one Python function each (same names)
# ---------------------------------------------------------------------------

def _check(h, rc):
    if rc != OK:
        msg = load().dbm_last_error(h).decode() if h else ""
        raise DbmError(rc, msg)


def dbm_init(params: dbm_params) -> int:
    L = load()
    h = C.c_void_p()
    rc = L.dbm_init(C.byref(params), C.byref(h))
    if rc != OK:
        raise DbmError(rc, L.dbm_init_error().decode())
    return h.value


def dbm_equilibrium_matrix(h, species: int) -> np.ndarray:
    out = np.zeros((Q, Q))
    _check(h, load().dbm_equilibrium_matrix(h, int(species), out.ctypes.data))
    return out


def dbm_get_layout(h) -> dbm_layout:
    out = dbm_layout()
    _check(h, load().dbm_get_layout(h, C.byref(out)))
    return out


def dbm_state_bytes(h) -> int:
    v = C.c_size_t()
    _check(h, load().dbm_state_bytes(h, C.byref(v)))
    return v.value


def dbm_scratch_bytes(h) -> int:
    v = C.c_size_t()
    _check(h, load().dbm_scratch_bytes(h, C.byref(v)))
    return v.value


def dbm_bind(h, f_a: int, f_b: int, scratch: int) -> None:
    _check(h, load().dbm_bind(h, f_a, f_b, scratch))


def dbm_set_state(h, rho_s: int, ux: int, uy: int, T: int, stream: int = 0) -> None:
    _check(h, load().dbm_set_state(h, rho_s, ux, uy, T, stream))


def dbm_set_f(h, f: int, stream: int = 0) -> None:
    _check(h, load().dbm_set_f(h, f, stream))


def dbm_get_f(h, f: int, stream: int = 0) -> None:
    _check(h, load().dbm_get_f(h, f, stream))


def dbm_step(h, nsteps: int, stream: int = 0) -> None:
    _check(h, load().dbm_step(h, int(nsteps), stream))


def dbm_moments(h, out: int, stream: int = 0) -> None:
    _check(h, load().dbm_moments(h, out, stream))


def dbm_nonequilibrium(h, out: int, stream: int = 0) -> None:
    _check(h, load().dbm_nonequilibrium(h, out, stream))


def dbm_conservation(h, out: int, stream: int = 0) -> None:
    _check(h, load().dbm_conservation(h, out, stream))


def dbm_conservation_noalloc(h, state: int, out: int, stream: int = 0) -> None:
    """Conserved totals without a scratch buffer (see include/dbm.h);
    state = 0 means the handle's current bound state."""
    _check(h, load().dbm_conservation_noalloc(h, state or None, out, stream))


def dbm_status(h, stream: int = 0) -> tuple[int, int]:
    bits = C.c_uint()
    rc = load().dbm_status(h, stream, C.byref(bits))
    return rc, bits.value


def dbm_steps_taken(h) -> int:
    return load().dbm_steps_taken(h)


def dbm_step_tile(h) -> tuple[int, int, int]:
    """(tile_x, tile_y, cells_per_thread) of the step's shared-memory tile;
    (0, 0, 0) when the step runs a kernel without one."""
    tx, ty, cw = C.c_int(), C.c_int(), C.c_int()
    _check(h, load().dbm_step_tile(h, C.byref(tx), C.byref(ty), C.byref(cw)))
    return tx.value, ty.value, cw.value


def dbm_last_error(h) -> str:
    return load().dbm_last_error(h).decode()


def dbm_destroy(h) -> None:
    load().dbm_destroy(h)


# ---------------------------------------------------------------------------
# convenience: a solver whose buffers are torch tensors on one device
# ---------------------------------------------------------------------------

class Solver:
    """One DBM problem on one GPU: the handle, two state buffers and the
    scratch buffer (torch allocations), and FP64 field transfers."""

    def __init__(self, problem, precision="fp64", device="cuda", stream=None, step_kernel="auto", **opts):
        """``opts`` are further dbm_params fields (make_params keywords)."""
        import torch

        self.torch = torch
        self.pb = problem
        self.device = torch.device(device)
        self.params = params_from_problem(problem, precision, step_kernel, **opts)
        self.h = dbm_init(self.params)
        self.layout = dbm_get_layout(self.h)
        nb = dbm_state_bytes(self.h)
        ns = dbm_scratch_bytes(self.h)
        self.buf = [torch.empty(nb, dtype=torch.uint8, device=self.device) for _ in range(2)]
        self.scratch = torch.zeros(ns, dtype=torch.uint8, device=self.device)
        dbm_bind(self.h, self.buf[0].data_ptr(), self.buf[1].data_ptr(), self.scratch.data_ptr())
        self.stream = stream
        self._uses(*self.buf, self.scratch)

    @property
    def S(self) -> int:
        return self.pb.ns

    @property
    def cells(self) -> int:
        return self.pb.nx * self.pb.ny

    def _st(self) -> int:
        """The stream the library works on.  With a stream of its own, the
        solver first waits for the caller's current stream (inputs it
        prepared) and the caller's stream waits for the solver's work before
        it reads any output (see _join)."""
        torch = self.torch
        if self.stream is None:
            return torch.cuda.current_stream(self.device).cuda_stream
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        return self.stream.cuda_stream

    def _uses(self, *tensors):
        # memory that the solver's own stream reads or writes is not handed
        # back to the allocator before that stream's work is done
        if self.stream is not None:
            for t in tensors:
                t.record_stream(self.stream)

    def _join(self):
        if self.stream is not None:
            self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _dev(self, a):
        torch = self.torch
        if isinstance(a, torch.Tensor):
            return a.to(device=self.device, dtype=torch.float64).contiguous()
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device)

    def set_state(self, rho_s=None, ux=None, uy=None, T=None):
        pb = self.pb
        rho_s = self._dev(pb.rho_s if rho_s is None else rho_s)
        ux = self._dev(pb.ux if ux is None else ux)
        uy = self._dev(pb.uy if uy is None else uy)
        T = self._dev(pb.T if T is None else T)
        assert rho_s.numel() == self.S * self.cells and ux.numel() == self.cells
        self._keep = (rho_s, ux, uy, T)
        self._uses(*self._keep)
        dbm_set_state(self.h, rho_s.data_ptr(), ux.data_ptr(), uy.data_ptr(), T.data_ptr(), self._st())

    def set_f(self, f):
        f = self._dev(f)
        assert f.numel() == self.S * Q * self.cells
        self._keep = (f,)
        self._uses(f)
        dbm_set_f(self.h, f.data_ptr(), self._st())

    def get_f(self):
        torch = self.torch
        out = torch.empty((self.S, Q, self.pb.ny, self.pb.nx), dtype=torch.float64, device=self.device)
        dbm_get_f(self.h, out.data_ptr(), self._st())
        self._join()
        return out

    def step(self, nsteps: int = 1):
        dbm_step(self.h, nsteps, self._st())

    def moments(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty((4 * self.S + 5, self.pb.ny, self.pb.nx), dtype=torch.float64,
                              device=self.device)
        dbm_moments(self.h, out.data_ptr(), self._st())
        self._join()
        return out

    def nonequilibrium(self):
        torch = self.torch
        out = torch.empty((20 * self.S, self.pb.ny, self.pb.nx), dtype=torch.float64, device=self.device)
        dbm_nonequilibrium(self.h, out.data_ptr(), self._st())
        self._join()
        return out

    def conservation(self):
        torch = self.torch
        out = torch.empty(self.S + 4, dtype=torch.float64, device=self.device)
        dbm_conservation(self.h, out.data_ptr(), self._st())
        self._join()
        return out

    def status(self):
        return dbm_status(self.h, self._st())

    def step_tile(self):
        """(tile_x, tile_y, cells_per_thread) of the step kernel; zeros when
        it has no shared-memory tile."""
        return dbm_step_tile(self.h)

    def close(self):
        if self.h:
            dbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------

def _bcheck(b, rc):
    if rc != OK:
        raise DbmError(rc, load().dbm_batch_last_error(b).decode() if b else "")


def dbm_batch_table_bytes(handles) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    v = C.c_size_t()
    rc = load().dbm_batch_table_bytes(arr, len(handles), C.byref(v))
    if rc != OK:
        raise DbmError(rc, "batch: handles must be bound FP32 handles with the same S <= 4")
    return v.value


def dbm_batch_create(handles, table: int, table_bytes: int, stream: int = 0) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    b = C.c_void_p()
    rc = load().dbm_batch_create(arr, len(handles), table, table_bytes, stream, C.byref(b))
    if rc != OK:
        raise DbmError(rc, "batch: handles must be bound FP32 handles with the same S <= 4")
    return b.value


def dbm_batch_tune(b, stream: int = 0, reps: int = 3) -> None:
    _bcheck(b, load().dbm_batch_tune(b, stream, reps))


def dbm_batch_step(b, nsteps: int, stream: int = 0) -> None:
    _bcheck(b, load().dbm_batch_step(b, int(nsteps), stream))


def dbm_batch_info(b) -> dict:
    v = [C.c_int() for _ in range(4)]
    _bcheck(b, load().dbm_batch_info(b, *[C.byref(x) for x in v]))
    return {"tile": (v[0].value, v[1].value), "tiles": v[2].value, "ctas": v[3].value}


def dbm_batch_get_config(b) -> dict:
    v = [C.c_int() for _ in range(5)]
    _bcheck(b, load().dbm_batch_get_config(b, *[C.byref(x) for x in v]))
    return {"tile": (v[0].value, v[1].value), "cells": v[2].value, "persistent": v[3].value, "promote": v[4].value}


def dbm_batch_set_config(b, tile, cells: int, persistent: int, promote: int, stream: int = 0) -> None:
    _bcheck(b, load().dbm_batch_set_config(b, int(tile[0]), int(tile[1]), int(cells), int(persistent), int(promote),
                                           stream))


def dbm_batch_destroy(b) -> None:
    load().dbm_batch_destroy(b)


class Batch:
    """Solvers (FP32, same species count) stepped together: one launch per
    step and chunk of instances, pairs of steps replayed from a CUDA graph.
    The kernel configuration is tuned (``tune``), given (``config``, a dict
    as returned by ``config()``), or the library's default."""

    def __init__(self, solvers, stream=None, tune=True, config=None):
        import torch

        self.torch = torch
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        handles = [s.h for s in self.solvers]
        nb = dbm_batch_table_bytes(handles)
        self.table = torch.empty(nb + 128, dtype=torch.uint8, device=dev)
        base = self.table.data_ptr()
        self._tp = (base + 127) // 128 * 128
        self.table.record_stream(self.stream)
        cur = torch.cuda.current_stream(dev)
        self._others = []
        for st in [cur] + [s.stream for s in self.solvers]:
            if st is not None and st != self.stream and all(st != o for o in self._others):
                self._others.append(st)
        self._enter()
        self.b = dbm_batch_create(handles, self._tp, nb, self.stream.cuda_stream)
        if config is not None:
            dbm_batch_set_config(self.b, config["tile"], config.get("cells", 1), config["persistent"], config["promote"],
                                 stream=self.stream.cuda_stream)
        elif tune:
            dbm_batch_tune(self.b, self.stream.cuda_stream)
        self._leave()

    def _enter(self):
        # the batch stream starts after the work queued on the caller's and
        # the solvers' streams, which continue only after the batch's steps
        for st in self._others:
            self.stream.wait_stream(st)

    def _leave(self):
        for st in self._others:
            st.wait_stream(self.stream)

    def step(self, nsteps: int):
        self._enter()
        dbm_batch_step(self.b, nsteps, self.stream.cuda_stream)
        self._leave()

    def info(self) -> dict:
        return dbm_batch_info(self.b)

    def config(self) -> dict:
        return dbm_batch_get_config(self.b)

    def close(self):
        if self.b:
            dbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
