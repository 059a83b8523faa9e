"""FP64 CPU oracle for the checkerboard Heisenberg spin-glass sweep.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs are the only callers.  The CUDA
library and its Python binding never import this package.

This module is a thin ctypes layer over ``hsg_oracle.c`` (plain C, double
precision).  Arrays are numpy float64, site-major: ``s[3*i + a]`` and
``J[3*i + d]`` with ``i = x + y*L + z*L*L`` (the paper's indexing, Sec. 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsg_oracle.c")
_LIB = os.path.join(_HERE, "libhsg_oracle.so")

OR, MET, HB, MET_OR = 0, 1, 2, 3
PROP_SPHERE, PROP_BALL = 0, 1
KIND_INIT, KIND_JGEN, KIND_MET, KIND_HB = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no target flags);
    with OpenMP where the compiler has it (only the timed CPU baseline uses
    more than one thread; results do not depend on the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("key", ctypes.c_uint32 * 2),
        ("sweep", ctypes.c_uint64),
        ("beta", ctypes.c_double),
        ("step", ctypes.c_double),
        ("hits", ctypes.c_int),
        ("proposal", ctypes.c_int),
    ]


class _Schedule(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("hits", ctypes.c_int),
        ("proposal", ctypes.c_int),
        ("step", ctypes.c_double),
        ("n_or", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("renorm_every", ctypes.c_int),
        ("energy_every", ctypes.c_int),
    ]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def _load():
    """The compiled oracle; HSG_ORACLE_LIB names another build of the same
    source to load instead (the mutation tests plant mistakes in copies)."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.environ.get("HSG_ORACLE_LIB") or build())
        lib.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.oracle_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u32p]
        lib.oracle_counter.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _u32p]
        lib.oracle_u01.argtypes = [ctypes.c_uint32]
        lib.oracle_u01.restype = ctypes.c_double
        lib.oracle_colour.argtypes = [ctypes.c_int, ctypes.c_int64]
        lib.oracle_init_spins.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _dp]
        lib.oracle_gaussian_couplings.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, _dp]
        lib.oracle_init_spin_sites.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u32p,
                                               ctypes.c_int, _dp]
        lib.oracle_gaussian_coupling_sites.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _u32p, ctypes.c_int, _dp]
        lib.oracle_local_field.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int64, _dp]
        lib.oracle_local_field_nb.argtypes = [_dp, _dp, _dp]
        lib.oracle_energy.argtypes = [ctypes.c_int, _dp, _dp]
        lib.oracle_energy.restype = ctypes.c_double
        lib.oracle_update_site.argtypes = [ctypes.c_int, _dp, _dp, ctypes.POINTER(_Params), ctypes.c_uint32,
                                           ctypes.c_int, _dp, _dp]
        lib.oracle_half_sweep.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_Params), _dp]
        lib.oracle_half_sweep_range.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_int64, _dp]
        lib.oracle_renorm.argtypes = [ctypes.c_int, _dp]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_sweeps.argtypes = [ctypes.c_int, _dp, _dp, ctypes.POINTER(_Schedule), _u32p, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_uint64), _dp, ctypes.POINTER(ctypes.c_int)]
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Threads of the half-sweep loops (1 by default)."""
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    """Processors the OpenMP build can use (1 without OpenMP)."""
    return int(_load().oracle_max_threads())


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


@dataclass
class Params:
    """Parameters of a half-sweep (key, sweep counter, beta, proposal)."""
    key: tuple = (0, 0)
    sweep: int = 0
    beta: float = 1.0
    step: float = 0.5
    hits: int = 1
    proposal: int = PROP_SPHERE

    def c(self) -> _Params:
        p = _Params()
        p.key[0], p.key[1] = int(self.key[0]), int(self.key[1])
        p.sweep, p.beta, p.step = int(self.sweep), float(self.beta), float(self.step)
        p.hits, p.proposal = int(self.hits), int(self.proposal)
        return p


@dataclass
class Schedule:
    """A sweep schedule: main update (None/MET/HB), OR sweeps, cadences."""
    kind: int = -1
    hits: int = 1
    proposal: int = PROP_SPHERE
    step: float = 0.5
    n_or: int = 0
    beta: float = 1.0
    renorm_every: int = 0
    energy_every: int = 0

    def c(self) -> _Schedule:
        s = _Schedule()
        s.kind, s.hits, s.proposal = int(self.kind), int(self.hits), int(self.proposal)
        s.step, s.n_or, s.beta = float(self.step), int(self.n_or), float(self.beta)
        s.renorm_every, s.energy_every = int(self.renorm_every), int(self.energy_every)
        return s


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def _stream_ok(rc: int, sample: int, replica: int) -> None:
    if rc != 0:
        raise ValueError(f"(sample {sample}, replica {replica}) outside the key's range: replica must be 0 or 1 "
                         "and sample < 2**31 (the stream number 2*sample + replica must name each pair once)")


def key(seed: int, sample: int = 0, replica: int = 0) -> tuple:
    lib = _load()
    k = (ctypes.c_uint32 * 2)()
    _stream_ok(lib.oracle_key(int(seed), int(sample), int(replica), k), sample, replica)
    return (int(k[0]), int(k[1]))


def counter(site: int, sweep: int, kind: int, colour: int, hit: int) -> tuple:
    lib = _load()
    c = (ctypes.c_uint32 * 4)()
    lib.oracle_counter(int(site), int(sweep), int(kind), int(colour), int(hit), c)
    return tuple(int(v) for v in c)


def u01(r: int) -> float:
    return _load().oracle_u01(int(r) & 0xFFFFFFFF)


def colour(L: int, i: int) -> int:
    return _load().oracle_colour(int(L), int(i))


def init_spins(L: int, seed: int, sample: int = 0, replica: int = 0) -> np.ndarray:
    s = np.zeros(3 * L ** 3, dtype=np.float64)
    _stream_ok(_load().oracle_init_spins(int(L), int(seed), int(sample), int(replica), _d(s)), sample, replica)
    return s


def gaussian_couplings(L: int, seed: int, sample: int = 0) -> np.ndarray:
    """J ~ N(0,1) from Philox (kind JGEN) and Box-Muller, site-major."""
    J = np.zeros(3 * L ** 3, dtype=np.float64)
    _stream_ok(_load().oracle_gaussian_couplings(int(L), int(seed), int(sample), _d(J)), sample, 0)
    return J


def init_spin_sites(sites, seed: int, sample: int = 0, replica: int = 0) -> np.ndarray:
    """Initial spins (n, 3) of listed site-major indices (any lattice size)."""
    idx = np.ascontiguousarray(np.asarray(sites, dtype=np.uint32).reshape(-1))
    out = np.zeros(3 * idx.size, dtype=np.float64)
    rc = _load().oracle_init_spin_sites(int(seed), int(sample), int(replica),
                                        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), idx.size, _d(out))
    _stream_ok(rc, sample, replica)
    return out.reshape(-1, 3)


def gaussian_coupling_sites(sites, seed: int, sample: int = 0) -> np.ndarray:
    """+x/+y/+z couplings (n, 3) of listed site-major indices (any lattice size)."""
    idx = np.ascontiguousarray(np.asarray(sites, dtype=np.uint32).reshape(-1))
    out = np.zeros(3 * idx.size, dtype=np.float64)
    rc = _load().oracle_gaussian_coupling_sites(int(seed), int(sample),
                                                idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), idx.size, _d(out))
    _stream_ok(rc, sample, 0)
    return out.reshape(-1, 3)


def local_field(L: int, J: np.ndarray, s: np.ndarray, i: int) -> np.ndarray:
    h = np.zeros(3, dtype=np.float64)
    _load().oracle_local_field(int(L), _d(J), _d(s), int(i), _d(h))
    return h


def local_field_nb(nb: np.ndarray, Jb: np.ndarray) -> np.ndarray:
    """Eq. 2 from explicit neighbours: nb (6, 3) spins at +x, -x, +y, -y, +z,
    -z and Jb (6,) the bonds to them (oracle_local_field's order)."""
    nb = np.ascontiguousarray(nb, dtype=np.float64).reshape(18)
    Jb = np.ascontiguousarray(Jb, dtype=np.float64).reshape(6)
    h = np.zeros(3, dtype=np.float64)
    _load().oracle_local_field_nb(_d(nb), _d(Jb), _d(h))
    return h


def energy(L: int, J: np.ndarray, s: np.ndarray) -> float:
    """Total energy E (Eq. 1, each bond once)."""
    return _load().oracle_energy(int(L), _d(J), _d(s))


def update_site(upd: int, s3, h3, params: Params, site: int, colour_: int):
    """One site update; returns (new spin, Metropolis margin)."""
    s = np.ascontiguousarray(s3, dtype=np.float64)
    h = np.ascontiguousarray(h3, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    m = ctypes.c_double(0.0)
    p = params.c()
    _load().oracle_update_site(int(upd), _d(s), _d(h), ctypes.byref(p), int(site), int(colour_), _d(out),
                               ctypes.byref(m))
    return out, m.value


def half_sweep(L: int, J: np.ndarray, s: np.ndarray, upd: int, colour_: int, params: Params,
               want_margins: bool = False):
    """In-place half-sweep of one colour; returns margins (or None)."""
    p = params.c()
    if want_margins:
        m = np.zeros(L ** 3, dtype=np.float64)
        _load().oracle_half_sweep(int(L), _d(J), _d(s), int(upd), int(colour_), ctypes.byref(p), _d(m))
        return m
    _load().oracle_half_sweep(int(L), _d(J), _d(s), int(upd), int(colour_), ctypes.byref(p), None)
    return None


def half_sweep_range(L: int, J: np.ndarray, s: np.ndarray, upd: int, colour_: int, params: Params, i0: int,
                     i1: int) -> None:
    """In-place half-sweep of the sites i0 <= i < i1 of one colour."""
    p = params.c()
    _load().oracle_half_sweep_range(int(L), _d(J), _d(s), int(upd), int(colour_), ctypes.byref(p), int(i0), int(i1),
                                    None)


def renorm(L: int, s: np.ndarray) -> None:
    _load().oracle_renorm(int(L), _d(s))


def sweeps(L: int, J: np.ndarray, s: np.ndarray, schedule: Schedule, key_: tuple, n_sweeps: int,
           sweep: int = 0):
    """In-place sweeps; returns (new sweep counter, energy log E/N)."""
    sc = schedule.c()
    k = (ctypes.c_uint32 * 2)(int(key_[0]), int(key_[1]))
    sw = ctypes.c_uint64(int(sweep))
    n_e = ctypes.c_int(0)
    cap = n_sweeps // schedule.energy_every + 1 if schedule.energy_every > 0 else 1
    elog = np.zeros(cap, dtype=np.float64)
    _load().oracle_sweeps(int(L), _d(J), _d(s), ctypes.byref(sc), k, int(n_sweeps), ctypes.byref(sw), _d(elog),
                          ctypes.byref(n_e))
    return int(sw.value), elog[: n_e.value].copy()
