"""ctypes binding of the C ABI in include/bp.h (argument marshalling only).

The functions keep the C names (``bp_create``, ``bp_step`` ...); ``Context``
bundles them for convenience.  Device memory comes from PyTorch's caching
allocator through the ``bp_allocator`` callbacks, and work goes on the
current PyTorch CUDA stream.  There is no CPU fallback: if the shared library
has not been built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bp.h")

BP_OK, BP_ERR_ARG, BP_ERR_OOM, BP_ERR_CUDA, BP_ERR_CFL = 0, -1, -2, -3, -4
BP_ERR_NONFINITE, BP_ERR_DOMAIN, BP_ERR_TIMEOUT, BP_ERR_IO, BP_ERR_STATE = -5, -6, -7, -8, -9
BP_PERIODIC, BP_OPEN = 0, 1
BP_DEPOSIT_ATOMIC, BP_DEPOSIT_SORTED = 0, 1
BP_TWO_BODY, BP_FREE = 0, 1
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)

STATUS_NAMES = {0: "BP_OK", -1: "BP_ERR_ARG", -2: "BP_ERR_OOM", -3: "BP_ERR_CUDA", -4: "BP_ERR_CFL",
                -5: "BP_ERR_NONFINITE", -6: "BP_ERR_DOMAIN", -7: "BP_ERR_TIMEOUT", -8: "BP_ERR_IO",
                -9: "BP_ERR_STATE"}


class BPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("dims", C.c_int), ("n", C.c_int64 * 3), ("dx", C.c_double * 3), ("dt", C.c_double),
                ("boundary", C.c_int * 3), ("deposit_mode", C.c_int), ("tile", C.c_int * 3)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class SpeciesDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("Zb", C.c_double), ("qc", C.c_double), ("mc", C.c_double),
                ("q", C.c_double), ("m", C.c_double), ("weight", C.c_double), ("lambda0_m", C.c_double),
                ("omega_b", C.POINTER(C.c_double)), ("n_omega", C.c_int)]


class LaserDesc(C.Structure):
    _fields_ = [("comp", C.c_int), ("a0", C.c_double), ("omega", C.c_double), ("theta", C.c_double),
                ("waist", C.c_double), ("fwhm", C.c_double), ("t0", C.c_double), ("ramp", C.c_double),
                ("phase", C.c_double), ("ia", C.c_int64), ("yc", C.c_double), ("zc", C.c_double)]


_lib: Optional[C.CDLL] = None
_p, _i, _i64, _d = C.c_void_p, C.c_int, C.c_int64, C.c_double

_SIGS = {
    "bp_create": (_i, [C.POINTER(GridDesc), C.POINTER(Allocator), _p, C.POINTER(_p)]),
    "bp_destroy": (None, [_p]),
    "bp_last_error": (C.c_char_p, [_p]),
    "bp_add_species": (_i, [_p, C.POINTER(SpeciesDesc), C.POINTER(_i)]),
    "bp_load_particles": (_i, [_p, _i, _p, _p, _p, _i64]),
    "bp_set_medium": (_i, [_p, _i, _p, _p, _i, C.c_uint64, _d]),
    "bp_add_laser": (_i, [_p, C.POINTER(LaserDesc)]),
    "bp_add_probe": (_i, [_p, _i, _p, _i64, _i64, C.POINTER(_i)]),
    "bp_step": (_i, [_p, _i64]),
    "bp_sync": (_i, [_p]),
    "bp_read_field": (_i, [_p, _i, _p, _i]),
    "bp_write_field": (_i, [_p, _i, _p, _i]),
    "bp_read_probe": (_i, [_p, _i, _p, _i64, C.POINTER(_i64)]),
    "bp_read_particles": (_i, [_p, _i, _p, _p, _p, _p, _i64, C.POINTER(_i64)]),
    "bp_read_particles_by_id": (_i, [_p, _i, _p, _i64, _p, _p, _p, _p, _p]),
    "bp_set_lattice": (_i, [_p, _i, _p, _i64, _i, C.c_double, C.c_uint64, C.c_double, _p]),
    "bp_save": (_i, [_p, C.c_char_p]),
    "bp_load": (_i, [_p, C.c_char_p]),
    "bp_residual": (_i, [_p, _p, _i]),
    "bp_residual_noalloc": (_i, [_p, _p]),
    "bp_reset": (_i, [_p]),
    "bp_set_omega": (_i, [_p, _i, _p, _i]),
    "bp_forward_ckpt": (_i, [_p, _i64, _i]),
    "bp_backward": (_i, [_p, _i, _p, _i, _p, _p, _i64, _p]),
    "bp_kernel_launches": (_i64, [_p]),
    "bp_time_push": (_i, [_p, _i]),
    "bp_set_record_capacity": (_i, [_p, C.c_int64]),
    "bp_read_field_async": (_i, [_p, _i, _p]),
    "bp_push_time": (_i, [_p, C.POINTER(_d), C.POINTER(_i64)]),
    "bp_push_work": (_i, [_p, C.POINTER(_i64), C.POINTER(_i64)]),
    "bp_field_work": (_i, [_p, C.POINTER(_i64), C.POINTER(_i64)]),
}


def header_functions() -> list[str]:
    """Names of the functions declared in include/bp.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_0-9]+\s*\*?\s*(bp_[a-z_0-9]+)\s*\(", txt, re.M)))


def lib() -> C.CDLL:
    """Load the CUDA library; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing ({LIB_PATH}); run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(int(a))


class _TorchAllocator:
    """bp_allocator backed by torch.cuda's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))
            except Exception:
                return None

        def _free(ptr, stream, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


class Context:
    """One simulation: grid, species, lasers, probes (see include/bp.h)."""

    def __init__(self, dims: int, n: Sequence[int], dx: Sequence[float], dt: float, boundary: Sequence[int],
                 deposit_mode: int = BP_DEPOSIT_SORTED, tile: Optional[Sequence[int]] = None,
                 stream: Optional[int] = None, allocator: str = "torch"):
        L = lib()
        self._L = L
        g = GridDesc()
        g.dims = dims
        for a in range(3):
            g.n[a] = int(n[a]) if a < dims else 1
            g.dx[a] = float(dx[a]) if a < dims else 1.0
            g.boundary[a] = int(boundary[a]) if a < dims else 0
            g.tile[a] = int(tile[a]) if (tile is not None and a < dims and tile[a]) else 0
        g.dt = float(dt)
        g.deposit_mode = deposit_mode
        self.dims = dims
        self.n = tuple(g.n[a] for a in range(3))
        self.dt = dt
        self._alloc = None
        ap = None
        if stream is None or allocator == "torch":
            import torch
            dev = torch.cuda.current_device()
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            if allocator == "torch":
                self._alloc = _TorchAllocator(dev)
                ap = C.pointer(self._alloc.struct)
        if hasattr(allocator, "struct"):  # a caller-built bp_allocator (kept alive by the context)
            self._alloc = allocator
            ap = C.pointer(allocator.struct)
        self.stream = stream
        h = C.c_void_p()
        rc = L.bp_create(C.byref(g), ap, C.c_void_p(stream), C.byref(h))
        if rc != BP_OK:
            raise BPError(rc, "bp_create failed")
        self._h = h
        self._keep = []
        self.probes = {}

    # -- helpers ------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != BP_OK:
            msg = self._L.bp_last_error(self._h)
            raise BPError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.bp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -------------------------------------------------------------
    def add_two_body(self, Zb, qc, mc, weight, lambda0_m, omega_b) -> int:
        om = np.ascontiguousarray(np.atleast_1d(omega_b), dtype=np.float64)
        d = SpeciesDesc(BP_TWO_BODY, Zb, qc, mc, 0.0, 0.0, weight, lambda0_m,
                        om.ctypes.data_as(C.POINTER(C.c_double)), len(om))
        sid = C.c_int()
        self._check(self._L.bp_add_species(self._h, C.byref(d), C.byref(sid)), "bp_add_species")
        return sid.value

    def add_free(self, q, m, weight) -> int:
        d = SpeciesDesc(BP_FREE, 0.0, 0.0, 0.0, q, m, weight, 0.0, None, 0)
        sid = C.c_int()
        self._check(self._L.bp_add_species(self._h, C.byref(d), C.byref(sid)), "bp_add_species")
        return sid.value

    def load_particles(self, sid: int, x, u=None, pidx=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        pidx = None if pidx is None else np.ascontiguousarray(pidx, dtype=np.int32)
        self._check(self._L.bp_load_particles(self._h, sid, _ptr(x), _ptr(u), _ptr(pidx), len(x)),
                    "bp_load_particles")

    def set_medium(self, sid: int, lo, hi, ppc: int, seed: int, sigma_u: float = 0.0):
        lo3 = (C.c_int64 * 3)(*(list(lo) + [0] * (3 - len(lo))))
        hi3 = (C.c_int64 * 3)(*(list(hi) + [1] * (3 - len(hi))))
        self._check(self._L.bp_set_medium(self._h, sid, lo3, hi3, ppc, C.c_uint64(seed), sigma_u),
                    "bp_set_medium")

    def add_laser(self, comp, a0, omega=1.0, theta=0.0, waist=0.0, fwhm=0.0, t0=0.0, ramp=0.0, phase=0.0,
                  ia=2, yc=0.0, zc=0.0):
        d = LaserDesc(comp, a0, omega, theta, waist, fwhm, t0, ramp, phase, int(ia), yc, zc)
        self._check(self._L.bp_add_laser(self._h, C.byref(d)), "bp_add_laser")

    def add_probe(self, comp: int, nodes, capacity: int) -> int:
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        pid = C.c_int()
        self._check(self._L.bp_add_probe(self._h, comp, _ptr(nodes), len(nodes), capacity, C.byref(pid)),
                    "bp_add_probe")
        self.probes[pid.value] = (len(nodes), capacity)
        return pid.value

    # -- running ------------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._L.bp_step(self._h, int(n)), "bp_step")

    def sync(self):
        self._check(self._L.bp_sync(self._h), "bp_sync")

    def read_field(self, comp: int) -> np.ndarray:
        nx, ny, nz = self.n
        out = np.empty(nx * ny * nz, dtype=np.float32)
        self._check(self._L.bp_read_field(self._h, comp, _ptr(out), 0), "bp_read_field")
        return out.reshape(nz, ny, nx)

    def read_field_device(self, comp: int, dst_ptr: int):
        self._check(self._L.bp_read_field(self._h, comp, C.c_void_p(dst_ptr), 1), "bp_read_field")

    def write_field(self, comp: int, data):
        a = np.ascontiguousarray(data, dtype=np.float32).ravel()
        if a.size != self.n[0] * self.n[1] * self.n[2]:
            raise ValueError("field size mismatch")
        self._check(self._L.bp_write_field(self._h, comp, _ptr(a), 0), "bp_write_field")

    def fields(self) -> np.ndarray:
        return np.stack([self.read_field(c) for c in range(9)])

    def read_probe(self, pid: int) -> np.ndarray:
        npts, cap = self.probes[pid]
        out = np.empty(npts * cap, dtype=np.float32)
        n = C.c_int64()
        self._check(self._L.bp_read_probe(self._h, pid, _ptr(out), cap, C.byref(n)), "bp_read_probe")
        k = min(n.value, cap)
        return out[: k * npts].reshape(k, npts)

    def read_particles(self, sid: int, cap: int):
        x1, x2, u1, u2 = (np.zeros((cap, 3)) for _ in range(4))
        n = C.c_int64()
        self._check(self._L.bp_read_particles(self._h, sid, _ptr(x1), _ptr(x2), _ptr(u1), _ptr(u2), cap,
                                              C.byref(n)), "bp_read_particles")
        k = min(n.value, cap)
        return x1[:k], x2[:k], u1[:k], u2[:k]

    def set_lattice(self, sid: int, sites, per_site: int, jitter: float, seed: int, sigma_u: float = 0.0,
                    site_param=None):
        """bp_set_lattice: per_site ions at every site with seeded Gaussian jitter."""
        st = np.ascontiguousarray(sites, dtype=np.float64)
        if st.ndim == 1:
            st = st[:, None]
        sp = None if site_param is None else np.ascontiguousarray(site_param, dtype=np.int32)
        self._check(self._L.bp_set_lattice(self._h, sid, _ptr(st), st.shape[0], int(per_site), float(jitter),
                                           int(seed), float(sigma_u), _ptr(sp)), "bp_set_lattice")

    def save(self, path: str):
        """bp_save: the run's state to a file."""
        self._check(self._L.bp_save(self._h, os.fsencode(path)), "bp_save")

    def load(self, path: str):
        """bp_load: a saved state into this context (same grid and species)."""
        self._check(self._L.bp_load(self._h, os.fsencode(path)), "bp_load")

    def read_particles_by_id(self, sid: int, ids):
        """States of the particles with the given load ids: x1, x2, u1, u2
        [n][3] and found [n] (bool)."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        n = len(ids)
        x1, x2, u1, u2 = (np.zeros((n, 3)) for _ in range(4))
        found = np.zeros(n, dtype=np.uint8)
        self._check(self._L.bp_read_particles_by_id(self._h, sid, _ptr(ids), n, _ptr(x1), _ptr(x2), _ptr(u1),
                                                    _ptr(u2), _ptr(found)), "bp_read_particles_by_id")
        return x1, x2, u1, u2, found.astype(bool)

    def residual(self) -> np.ndarray:
        nx, ny, nz = self.n
        out = np.empty(nx * ny * nz, dtype=np.float64)
        self._check(self._L.bp_residual(self._h, _ptr(out), 0), "bp_residual")
        return out.reshape(nz, ny, nx)

    def residual_noalloc(self) -> np.ndarray:
        """bp_residual_noalloc: the residual through the library's static
        scratch (no device allocation during the call)."""
        nx, ny, nz = self.n
        out = np.empty(nx * ny * nz, dtype=np.float64)
        self._check(self._L.bp_residual_noalloc(self._h, _ptr(out)), "bp_residual_noalloc")
        return out.reshape(nz, ny, nx)

    def reset(self):
        self._check(self._L.bp_reset(self._h), "bp_reset")

    def set_omega(self, sid: int, omega_b):
        om = np.ascontiguousarray(np.atleast_1d(omega_b), dtype=np.float64)
        self._check(self._L.bp_set_omega(self._h, sid, _ptr(om), len(om)), "bp_set_omega")

    def forward_ckpt(self, nsteps: int, K: int):
        self._check(self._L.bp_forward_ckpt(self._h, int(nsteps), int(K)), "bp_forward_ckpt")

    def backward(self, pid: int, dl_dprobe, sid: int, n_omega: int, group=None, n_groups: int = 0):
        dl = np.ascontiguousarray(dl_dprobe, dtype=np.float32)
        go = np.zeros(n_omega)
        gg = np.zeros((max(n_groups, 1), self.dims))
        grp = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
        self._check(self._L.bp_backward(self._h, pid, _ptr(dl), sid, _ptr(go), _ptr(grp), int(n_groups),
                                        _ptr(gg) if group is not None else None), "bp_backward")
        return go, gg[:n_groups]

    def kernel_launches(self) -> int:
        return int(self._L.bp_kernel_launches(self._h))

    def read_field_async(self, comp: int, dst) -> None:
        """Enqueue a read of field comp into dst (a contiguous float32 array
        of the grid's size, ideally page-locked); valid after sync()."""
        self._check(self._L.bp_read_field_async(self._h, comp, _ptr(dst)), "bp_read_field_async")

    def set_record_capacity(self, n: int):
        self._check(self._L.bp_set_record_capacity(self._h, int(n)), "bp_set_record_capacity")

    def time_push(self, enable: bool):
        self._check(self._L.bp_time_push(self._h, int(enable)), "bp_time_push")

    def push_time(self):
        ms = C.c_double()
        n = C.c_int64()
        self._check(self._L.bp_push_time(self._h, C.byref(ms), C.byref(n)), "bp_push_time")
        return ms.value, n.value

    def push_work(self):
        """(full pushes, quiet drifts) of the timed push launches (bp_push_work)."""
        full = C.c_int64()
        quiet = C.c_int64()
        self._check(self._L.bp_push_work(self._h, C.byref(full), C.byref(quiet)), "bp_push_work")
        return full.value, quiet.value

    def field_work(self):
        """(tiles the field kernels updated, summed over the steps; steps
        counted) since the last call (bp_field_work; zero on grids of fewer
        than 1024 tiles, where every tile is updated)."""
        tiles = C.c_int64()
        steps = C.c_int64()
        self._check(self._L.bp_field_work(self._h, C.byref(tiles), C.byref(steps)), "bp_field_work")
        return tiles.value, steps.value
