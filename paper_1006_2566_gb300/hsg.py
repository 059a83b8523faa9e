"""ctypes binding of libhsg (the C ABI in ``include/hsg.h``).

Argument marshalling only: every step of the Monte Carlo runs in the CUDA
kernels of ``libhsg.so``.  The functions keep the C names; ``Lattice`` wraps
a context for convenience.  Importing this module loads the library and
raises ``ImportError`` if it has not been built: there is no fallback.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the memory
space is passed to the library as ``HSG_HOST`` / ``HSG_DEVICE``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhsg.so")

HSG_OK, HSG_EINVAL, HSG_ENOMEM, HSG_ECUDA, HSG_ETIMEOUT, HSG_EBUSY = range(6)
HSG_NONE, HSG_METROPOLIS, HSG_HEATBATH, HSG_OVERRELAX, HSG_METROPOLIS_OR = range(5)
HSG_PROP_SPHERE, HSG_PROP_BALL = 0, 1
HSG_F32, HSG_F64 = 0, 1
HSG_HOST, HSG_DEVICE = 0, 1
HSG_KERNEL_AUTO, HSG_KERNEL_GLOBAL, HSG_KERNEL_SLAB, HSG_KERNEL_WAVE = 0, 1, 2, 3
HSG_LAYOUT_FLOAT4, HSG_LAYOUT_PACKED = 0, 1
(HSG_PROF_INIT, HSG_PROF_LAYOUT, HSG_PROF_OVERRELAX, HSG_PROF_METROPOLIS, HSG_PROF_HEATBATH,
 HSG_PROF_ENERGY, HSG_PROF_RENORM, HSG_PROF_OVERRELAX_RENORM, HSG_PROF_COUNT) = range(9)


class HsgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class hsg_schedule(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("hits", ctypes.c_int),
        ("proposal", ctypes.c_int),
        ("step", ctypes.c_float),
        ("n_or", ctypes.c_int),
        ("T", ctypes.c_double),
        ("renorm_every", ctypes.c_int),
        ("energy_every", ctypes.c_int),
        ("kernel", ctypes.c_int),
    ]


def schedule(kind=HSG_NONE, hits=1, proposal=HSG_PROP_SPHERE, step=0.5, n_or=0, T=1.0, renorm_every=0,
             energy_every=0, kernel=HSG_KERNEL_AUTO) -> hsg_schedule:
    """A filled ``hsg_schedule`` (T may be ``math.inf``)."""
    return hsg_schedule(int(kind), int(hits), int(proposal), float(step), int(n_or), float(T), int(renorm_every),
                        int(energy_every), int(kernel))


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)
_vp, _i, _u32, _u64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_sch_p = ctypes.POINTER(hsg_schedule)

_SIGS = {
    "hsg_create": ([ctypes.POINTER(_vp), _i, _u64, _u32, _u32, _vp], _i),
    "hsg_create_layout": ([ctypes.POINTER(_vp), _i, _u64, _u32, _u32, _vp, _i], _i),
    "hsg_destroy": ([_vp], _i),
    "hsg_set_couplings": ([_vp, _vp, _i, _i], _i),
    "hsg_generate_couplings": ([_vp], _i),
    "hsg_get_couplings": ([_vp, _vp, _i], _i),
    "hsg_sweep": ([_vp, _sch_p, _i], _i),
    "hsg_energy": ([_vp, ctypes.POINTER(_d)], _i),
    "hsg_get_energy_log": ([_vp, ctypes.POINTER(_d), _i, ctypes.POINTER(_i)], _i),
    "hsg_clear_energy_log": ([_vp], _i),
    "hsg_get_spins": ([_vp, _vp, _i], _i),
    "hsg_set_spins": ([_vp, _vp, _i], _i),
    "hsg_get_sweep": ([_vp, ctypes.POINTER(_u64)], _i),
    "hsg_get_sites": ([_vp, _vp, _i, _vp, _vp], _i),
    "hsg_set_sweep": ([_vp, _u64], _i),
    "hsg_half_sweep": ([_vp, _sch_p, _i, _i], _i),
    "hsg_renorm": ([_vp], _i),
    "hsg_kernel_for": ([_vp, _sch_p, ctypes.POINTER(_i)], _i),
    "hsg_profile": ([_vp, _i], _i),
    "hsg_profile_read": ([_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_u64)], _i),
    "hsg_profile_reset": ([_vp], _i),
    "hsg_launch_count": ([_vp, ctypes.POINTER(_u64)], _i),
    "hsg_last_error": ([_vp], ctypes.c_char_p),
    "hsg_status_string": ([_i], ctypes.c_char_p),
    "hsg_version": ([], _i),
    "hsg_philox": ([_u64, _u32, _u32, _u32, _u32, _u32, _u32, _vp, _vp], _i),
    "hsg_test_fail_alloc": ([_i], _i),
    "hsg_test_stall_tensor_loads": ([_i], _i),
    "hsg_energy_noalloc": ([_i, _vp, _vp, _vp, _vp], _i),
    "hsg_pool_create": ([ctypes.POINTER(_vp), _u64, _i, _vp], _i),
    "hsg_pool_destroy": ([_vp], _i),
    "hsg_pool_admit": ([_vp, _i, _u64, _u32, _u32, _d, _vp, _i, _i, ctypes.POINTER(_i)], _i),
    "hsg_pool_retire": ([_vp, _i], _i),
    "hsg_pool_sweep": ([_vp, _sch_p, _i], _i),
    "hsg_pool_energies": ([_vp, ctypes.POINTER(_d), _i], _i),
    "hsg_pool_energies_async": ([_vp, _i], _i),
    "hsg_pool_energies_read": ([_vp, _i, ctypes.POINTER(_d), _i], _i),
    "hsg_pool_energies_slots_async": ([_vp, _i, ctypes.POINTER(_i), _i], _i),
    "hsg_pool_get_spins": ([_vp, _i, _vp, _i], _i),
    "hsg_pool_get_sweep": ([_vp, _i, ctypes.POINTER(_u64)], _i),
    "hsg_pool_usage": ([_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_i)], _i),
    "hsg_pool_config": ([_vp, _i, _i, _i, _i], _i),
    "hsg_pool_autotune": ([_vp, _sch_p, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                           ctypes.POINTER(_i)], _i),
    "hsg_pool_launch_count": ([_vp, ctypes.POINTER(_u64)], _i),
    "hsg_pool_last_error": ([_vp], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _status_name(s: int) -> str:
    return _lib.hsg_status_string(int(s)).decode()


def _check(status: int, ctx=None) -> None:
    if status != HSG_OK:
        msg = _lib.hsg_last_error(ctx).decode()
        raise HsgError(status, msg)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _array_ptr(a, want_dtype=None):
    """(pointer, where, dtype code, n elements) of a numpy array or torch tensor."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        code = {torch.float32: HSG_F32, torch.float64: HSG_F64}.get(a.dtype)
        where = HSG_DEVICE if a.is_cuda else HSG_HOST
        return a.data_ptr(), where, code, a.numel()
    a = np.asarray(a)
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    code = {np.dtype(np.float32): HSG_F32, np.dtype(np.float64): HSG_F64}.get(a.dtype)
    return a.ctypes.data, HSG_HOST, code, a.size


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------

def hsg_create(L: int, seed: int, sample: int = 0, replica: int = 0, stream=None,
               layout: int = HSG_LAYOUT_FLOAT4) -> ctypes.c_void_p:
    if layout != HSG_LAYOUT_FLOAT4:
        return hsg_create_layout(L, seed, sample, replica, stream, layout)
    ctx = _vp()
    _check(_lib.hsg_create(ctypes.byref(ctx), int(L), int(seed), int(sample), int(replica), _stream_ptr(stream)))
    return ctx


def hsg_create_layout(L: int, seed: int, sample: int = 0, replica: int = 0, stream=None,
                      layout: int = HSG_LAYOUT_PACKED) -> ctypes.c_void_p:
    ctx = _vp()
    _check(_lib.hsg_create_layout(ctypes.byref(ctx), int(L), int(seed), int(sample), int(replica),
                                  _stream_ptr(stream), int(layout)))
    return ctx


def hsg_destroy(ctx) -> None:
    _check(_lib.hsg_destroy(ctx))


def hsg_set_couplings(ctx, J) -> None:
    ptr, where, code, n = _array_ptr(J)
    if code is None:
        raise TypeError("couplings must be float32 or float64")
    _check(_lib.hsg_set_couplings(ctx, ptr, code, where), ctx)


def hsg_generate_couplings(ctx) -> None:
    _check(_lib.hsg_generate_couplings(ctx), ctx)


def hsg_get_couplings(ctx, out) -> None:
    ptr, where, code, _ = _array_ptr(out)
    if code != HSG_F32:
        raise TypeError("couplings are read back as float32")
    _check(_lib.hsg_get_couplings(ctx, ptr, where), ctx)


def hsg_sweep(ctx, sched: hsg_schedule, n_sweeps: int) -> None:
    _check(_lib.hsg_sweep(ctx, ctypes.byref(sched), int(n_sweeps)), ctx)


def hsg_energy(ctx) -> float:
    e = _d(0.0)
    _check(_lib.hsg_energy(ctx, ctypes.byref(e)), ctx)
    return e.value


def hsg_get_energy_log(ctx) -> np.ndarray:
    n = _i(0)
    _check(_lib.hsg_get_energy_log(ctx, None, 0, ctypes.byref(n)), ctx)
    out = np.zeros(n.value, dtype=np.float64)
    if n.value:
        _check(_lib.hsg_get_energy_log(ctx, out.ctypes.data_as(ctypes.POINTER(_d)), n.value, ctypes.byref(n)), ctx)
    return out


def hsg_clear_energy_log(ctx) -> None:
    _check(_lib.hsg_clear_energy_log(ctx), ctx)


def hsg_get_spins(ctx, out) -> None:
    ptr, where, code, _ = _array_ptr(out)
    if code != HSG_F32:
        raise TypeError("spins are float32")
    _check(_lib.hsg_get_spins(ctx, ptr, where), ctx)


def hsg_set_spins(ctx, spins) -> None:
    ptr, where, code, _ = _array_ptr(spins)
    if code != HSG_F32:
        raise TypeError("spins are float32")
    _check(_lib.hsg_set_spins(ctx, ptr, where), ctx)


def hsg_get_sweep(ctx) -> int:
    v = _u64(0)
    _check(_lib.hsg_get_sweep(ctx, ctypes.byref(v)), ctx)
    return v.value


def hsg_set_sweep(ctx, sweep: int) -> None:
    _check(_lib.hsg_set_sweep(ctx, int(sweep)), ctx)


def hsg_half_sweep(ctx, sched: hsg_schedule, update: int, colour: int) -> None:
    _check(_lib.hsg_half_sweep(ctx, ctypes.byref(sched), int(update), int(colour)), ctx)


def hsg_renorm(ctx) -> None:
    _check(_lib.hsg_renorm(ctx), ctx)


def hsg_get_sites(ctx, sites, want_bonds: bool = True):
    """Spins (n, 3) and, if asked, +x/+y/+z bonds (n, 3) of site-major indices."""
    idx = np.ascontiguousarray(np.asarray(sites, dtype=np.uint32).reshape(-1))
    n = idx.size
    spins = np.empty((n, 3), dtype=np.float32)
    bonds = np.empty((n, 3), dtype=np.float32) if want_bonds else None
    _check(_lib.hsg_get_sites(ctx, idx.ctypes.data, n, spins.ctypes.data,
                              bonds.ctypes.data if want_bonds else None), ctx)
    return spins, bonds


def hsg_kernel_for(ctx, sched: hsg_schedule) -> int:
    """The HSG_KERNEL_* variant hsg_sweep runs for the OR sweeps of `sched`."""
    k = _i(0)
    _check(_lib.hsg_kernel_for(ctx, ctypes.byref(sched), ctypes.byref(k)), ctx)
    return k.value


def hsg_profile(ctx, on: bool) -> None:
    _check(_lib.hsg_profile(ctx, 1 if on else 0), ctx)


def hsg_profile_read(ctx, kclass: int):
    ms, n = _d(0.0), _u64(0)
    _check(_lib.hsg_profile_read(ctx, int(kclass), ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def hsg_profile_reset(ctx) -> None:
    _check(_lib.hsg_profile_reset(ctx), ctx)


def hsg_launch_count(ctx) -> int:
    v = _u64(0)
    _check(_lib.hsg_launch_count(ctx, ctypes.byref(v)), ctx)
    return v.value


def hsg_last_error(ctx=None) -> str:
    return _lib.hsg_last_error(ctx).decode()


def hsg_status_string(status: int) -> str:
    return _status_name(status)


def hsg_version() -> int:
    return _lib.hsg_version()


def hsg_philox(seed: int, sample: int, replica: int, c1: int, c2: int, c3: int, out, stream=None) -> None:
    ptr, where, _, n = _array_ptr(out)
    if where != HSG_DEVICE:
        raise ValueError("out must be a CUDA tensor of 4*n uint32 (int32) words")
    _check(_lib.hsg_philox(int(seed), int(sample), int(replica), int(c1), int(c2), int(c3), n // 4, ptr,
                           _stream_ptr(stream)))


def hsg_test_fail_alloc(k: int) -> None:
    _check(_lib.hsg_test_fail_alloc(int(k)))


def hsg_test_stall_tensor_loads(on) -> None:
    """True / 1: the couplings' tensor loads; 2: the colour-1 planes' barriers; 3: both; False / 0: off."""
    _check(_lib.hsg_test_stall_tensor_loads(int(on)))


def hsg_energy_noalloc(L: int, spins, J, e_out, stream=None) -> None:
    """E/N of caller-held device arrays (site-major fp32 spins and J) into the
    device double ``e_out``, queued on ``stream``; the library allocates
    nothing (see include/hsg.h for who needs this).

    The library cannot see the arrays' lengths, so they are checked here:
    float32 ``spins`` and ``J`` of at least 3 L^3 elements and a float64
    ``e_out`` of at least one, all CUDA tensors on the current device
    (ValueError otherwise).  An L outside [4, 1624] or odd goes to the
    library, which rejects it with HSG_EINVAL before launching anything."""
    import torch

    L = int(L)
    dev = torch.cuda.current_device()
    want = [("spins", spins, HSG_F32, 3 * L ** 3), ("J", J, HSG_F32, 3 * L ** 3), ("e_out", e_out, HSG_F64, 1)]
    ptrs = []
    for name, a, code_want, n_want in want:
        if not isinstance(a, torch.Tensor) or not a.is_cuda:
            raise ValueError(f"hsg_energy_noalloc: {name} must be a CUDA tensor")
        if a.device.index != dev:
            raise ValueError(f"hsg_energy_noalloc: {name} is on {a.device}, not the current device cuda:{dev}")
        ptr, _, code, n = _array_ptr(a)
        if code != code_want:
            raise ValueError(f"hsg_energy_noalloc: {name} must be {'float32' if code_want == HSG_F32 else 'float64'}")
        if L % 2 == 0 and 4 <= L <= 1624 and n < n_want:  # any other L: the library's HSG_EINVAL, no launch
            raise ValueError(f"hsg_energy_noalloc: {name} holds {n} elements, needs {n_want} for L = {L}")
        ptrs.append(ptr)
    _check(_lib.hsg_energy_noalloc(L, ptrs[0], ptrs[1], ptrs[2], _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class Lattice:
    """One L^3 lattice on the current CUDA device (a thin wrapper over a context)."""

    def __init__(self, L: int, seed: int, sample: int = 0, replica: int = 0, stream=None,
                 layout: int = HSG_LAYOUT_FLOAT4):
        self.L = int(L)
        self.N = self.L ** 3
        self.ctx = None
        self.ctx = hsg_create(L, seed, sample, replica, stream, layout)

    def close(self) -> None:
        if self.ctx is not None and self.ctx.value:
            hsg_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_couplings(self, J) -> None:
        hsg_set_couplings(self.ctx, J)

    def generate_couplings(self) -> None:
        hsg_generate_couplings(self.ctx)

    def couplings(self) -> np.ndarray:
        out = np.zeros(3 * self.N, dtype=np.float32)
        hsg_get_couplings(self.ctx, out)
        return out

    def sweep(self, sched: hsg_schedule, n_sweeps: int = 1) -> None:
        hsg_sweep(self.ctx, sched, n_sweeps)

    def half_sweep(self, sched: hsg_schedule, update: int, colour: int) -> None:
        hsg_half_sweep(self.ctx, sched, update, colour)

    def energy(self) -> float:
        return hsg_energy(self.ctx)

    def energy_log(self) -> np.ndarray:
        return hsg_get_energy_log(self.ctx)

    def spins(self) -> np.ndarray:
        out = np.zeros(3 * self.N, dtype=np.float32)
        hsg_get_spins(self.ctx, out)
        return out

    def set_spins(self, s) -> None:
        hsg_set_spins(self.ctx, s)

    def renorm(self) -> None:
        hsg_renorm(self.ctx)

    @property
    def sweep_count(self) -> int:
        return hsg_get_sweep(self.ctx)

    @sweep_count.setter
    def sweep_count(self, v: int) -> None:
        hsg_set_sweep(self.ctx, v)


# ---------------------------------------------------------------------------
# Pools (many lattices swept together)
# ---------------------------------------------------------------------------

def _pcheck(status: int, pool) -> None:
    if status != HSG_OK:
        raise HsgError(status, _lib.hsg_pool_last_error(pool).decode() or _lib.hsg_last_error(None).decode())


def hsg_pool_create(budget_bytes: int, max_slots: int, stream=None) -> ctypes.c_void_p:
    pool = _vp()
    _check(_lib.hsg_pool_create(ctypes.byref(pool), int(budget_bytes), int(max_slots), _stream_ptr(stream)))
    return pool


def hsg_pool_destroy(pool) -> None:
    _check(_lib.hsg_pool_destroy(pool))


def hsg_pool_admit(pool, L: int, seed: int, sample: int = 0, replica: int = 0, T: float = 1.0, J=None) -> int:
    """Admit a lattice; J None draws the couplings on the device.  Raises
    HsgError with status HSG_EBUSY when the pool is full."""
    slot = _i(-1)
    if J is None:
        ptr, code, where = None, HSG_F32, HSG_DEVICE
    else:
        ptr, where, code, _ = _array_ptr(J)
        if code is None:
            raise TypeError("couplings must be float32 or float64")
    _pcheck(_lib.hsg_pool_admit(pool, int(L), int(seed), int(sample), int(replica), float(T), ptr, code, where,
                                ctypes.byref(slot)), pool)
    return slot.value


def hsg_pool_retire(pool, slot: int) -> None:
    _pcheck(_lib.hsg_pool_retire(pool, int(slot)), pool)


def hsg_pool_sweep(pool, sched: hsg_schedule, n_sweeps: int) -> None:
    _pcheck(_lib.hsg_pool_sweep(pool, ctypes.byref(sched), int(n_sweeps)), pool)


def hsg_pool_energies(pool, n: int) -> np.ndarray:
    out = np.zeros(int(n), dtype=np.float64)
    _pcheck(_lib.hsg_pool_energies(pool, out.ctypes.data_as(ctypes.POINTER(_d)), int(n)), pool)
    return out


def hsg_pool_energies_async(pool, buffer: int) -> None:
    _pcheck(_lib.hsg_pool_energies_async(pool, int(buffer)), pool)


def hsg_pool_energies_slots_async(pool, buffer: int, slots) -> None:
    sl = np.ascontiguousarray(np.asarray(slots, dtype=np.int32).ravel())
    _pcheck(_lib.hsg_pool_energies_slots_async(pool, int(buffer), sl.ctypes.data_as(ctypes.POINTER(_i)), sl.size),
            pool)


def hsg_pool_energies_read(pool, buffer: int, n: int) -> np.ndarray:
    out = np.zeros(int(n), dtype=np.float64)
    _pcheck(_lib.hsg_pool_energies_read(pool, int(buffer), out.ctypes.data_as(ctypes.POINTER(_d)), int(n)), pool)
    return out


def hsg_pool_get_spins(pool, slot: int, out) -> None:
    ptr, where, code, _ = _array_ptr(out)
    if code != HSG_F32:
        raise TypeError("spins are float32")
    _pcheck(_lib.hsg_pool_get_spins(pool, int(slot), ptr, where), pool)


def hsg_pool_get_sweep(pool, slot: int) -> int:
    v = _u64(0)
    _pcheck(_lib.hsg_pool_get_sweep(pool, int(slot), ctypes.byref(v)), pool)
    return v.value


def hsg_pool_usage(pool):
    used, budget, active = _u64(0), _u64(0), _i(0)
    _pcheck(_lib.hsg_pool_usage(pool, ctypes.byref(used), ctypes.byref(budget), ctypes.byref(active)), pool)
    return used.value, budget.value, active.value


def hsg_pool_config(pool, threads: int, tile_sites: int, blocks_per_sm: int, hits_per_pass: int = 0) -> None:
    _pcheck(_lib.hsg_pool_config(pool, int(threads), int(tile_sites), int(blocks_per_sm), int(hits_per_pass)), pool)


def hsg_pool_autotune(pool, sched: hsg_schedule):
    """(threads, tile_sites, blocks_per_sm, hits_per_pass) chosen and set."""
    t, ts, b, h = _i(0), _i(0), _i(0), _i(0)
    _pcheck(_lib.hsg_pool_autotune(pool, ctypes.byref(sched), ctypes.byref(t), ctypes.byref(ts), ctypes.byref(b),
                                   ctypes.byref(h)), pool)
    return t.value, ts.value, b.value, h.value


def hsg_pool_launch_count(pool) -> int:
    v = _u64(0)
    _pcheck(_lib.hsg_pool_launch_count(pool, ctypes.byref(v)), pool)
    return v.value


def hsg_pool_last_error(pool) -> str:
    return _lib.hsg_pool_last_error(pool).decode()


class Pool:
    """Many lattices in one device arena (a thin wrapper over hsg_pool_*)."""

    def __init__(self, budget_bytes: int, max_slots: int, stream=None):
        self.pool = hsg_pool_create(budget_bytes, max_slots, stream)
        self.max_slots = int(max_slots)
        self.sides: dict[int, int] = {}

    def close(self) -> None:
        if self.pool is not None and self.pool.value:
            hsg_pool_destroy(self.pool)
        self.pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, L, seed, sample=0, replica=0, T=1.0, J=None) -> int:
        slot = hsg_pool_admit(self.pool, L, seed, sample, replica, T, J)
        self.sides[slot] = int(L)
        return slot

    def retire(self, slot: int) -> None:
        hsg_pool_retire(self.pool, slot)
        self.sides.pop(slot, None)

    def sweep(self, sched: hsg_schedule, n_sweeps: int = 1) -> None:
        hsg_pool_sweep(self.pool, sched, n_sweeps)

    def energies(self) -> np.ndarray:
        return hsg_pool_energies(self.pool, self.max_slots)

    def energies_async(self, buffer: int, slots=None) -> None:
        """Queue the E/N of every slot, or of the listed slots only, into
        pinned buffer 0 or 1 (no wait)."""
        if slots is None:
            hsg_pool_energies_async(self.pool, buffer)
        else:
            hsg_pool_energies_slots_async(self.pool, buffer, slots)

    def energies_read(self, buffer: int) -> np.ndarray:
        """Wait for the values queued into `buffer` and return them."""
        return hsg_pool_energies_read(self.pool, buffer, self.max_slots)

    def spins(self, slot: int) -> np.ndarray:
        out = np.zeros(3 * self.sides[slot] ** 3, dtype=np.float32)
        hsg_pool_get_spins(self.pool, slot, out)
        return out

    def sweep_count(self, slot: int) -> int:
        return hsg_pool_get_sweep(self.pool, slot)

    def usage(self):
        return hsg_pool_usage(self.pool)
