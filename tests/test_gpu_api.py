"""GPU tests of the library's lattice generator, state files and
asynchronous field reads: bp_set_lattice against the host definition of the
seeded lattice, bp_save / bp_load continuing a run bit for bit, and
bp_read_field_async returning each step's field as the synchronous read does."""
import os

import numpy as np
import pytest

from paper_2208_08038_gb300 import synth
from _common import field_rel_l2, gpu_from_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2208_08038_gb300 import binding
    binding.lib()


def bragg_small():
    return synth.bragg_2d(seed=5, n=256, cells_per_lambda=16, sites=(6, 6), waist_lambda=3.0,
                               fwhm_lambda=3.0, nb=0.05, steps=60)


def test_set_lattice_matches_host_definition():
    """The device lattice (positions with seeded jitter, thermal momenta, one
    parameter index per site) equals synth.lattice's, ion by ion."""
    from paper_2208_08038_gb300 import binding as B
    wl = bragg_small()
    sp = wl.species[0]
    m = wl.meta
    sites = synth.square_lattice(m["origin"], m["d"], m["sites"])
    per_site, jitter, sigma = 4, 0.05 * m["d"], 2e-3
    x_h, u_h = synth.lattice(77, sites, per_site, jitter, sigma)
    param = (np.arange(len(sites)) % 3).astype(np.int32)
    omega = np.array([3.0, 3.5, 4.0])
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, omega)
    ctx.set_lattice(sid, sites, per_site, jitter, 77, sigma, param)
    x1, x2, u1, u2 = ctx.read_particles(sid, len(x_h))
    assert len(x1) == len(x_h)
    assert np.abs(x1[:, :2] - x_h).max() < 1e-6 * wl.dx[0]
    assert np.array_equal(x1, x2)
    assert np.abs(u1 - u_h).max() < 1e-6 * np.abs(u_h).max()
    # the same run from the device lattice and from the host arrays
    ctx2 = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    sid2 = ctx2.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, omega)
    ctx2.load_particles(sid2, x_h, u_h, np.repeat(param, per_site))
    for c in (ctx, ctx2):
        for L in wl.lasers:
            c.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
        c.step(40)
        c.sync()
    assert field_rel_l2(ctx.fields(), ctx2.fields(), comps=range(9)) < 1e-6
    ctx.close()
    ctx2.close()


def small_periodic_3d():
    wl = synth.neutral_3d(seed=9, steps=30, n=(32, 16, 16), ppc=4, sigma_u=5e-2, margin=2)
    wl.bc = (0, 0, 0)
    wl.lasers[0].waist = 0.5 * synth.LAMBDA0
    wl.lasers[0].a0 = 0.05
    return wl


def test_save_load_continues_bit_exact(tmp_path):
    from paper_2208_08038_gb300 import binding as B
    wl = small_periodic_3d()
    path = os.path.join(tmp_path, "state.bp")
    a, sa, _ = gpu_from_workload(wl, deposit_mode=1)
    a.step(12)
    a.save(path)
    a.step(10)
    a.sync()
    fa = a.fields()
    pa = a.read_particles(sa[0], len(wl.species[0].x))
    # a fresh context with the same grid and species, not loaded
    sp = wl.species[0]
    b = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    sb = b.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    for L in wl.lasers:
        b.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    b.load(path)
    b.step(10)
    b.sync()
    assert np.array_equal(fa, b.fields())
    pb = b.read_particles(sb, len(sp.x))
    for qa, qb in zip(pa, pb):
        assert np.array_equal(qa, qb)
    a.close()
    b.close()


def test_load_rejects_other_grids_and_foreign_files(tmp_path):
    from paper_2208_08038_gb300 import binding as B
    wl = small_periodic_3d()
    path = os.path.join(tmp_path, "state.bp")
    a, _, _ = gpu_from_workload(wl, deposit_mode=1)
    a.save(path)
    sp = wl.species[0]
    other = B.Context(wl.D, (64, 16, 16), wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    other.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    with pytest.raises(B.BPError) as e:
        other.load(path)
    assert e.value.code == B.BP_ERR_ARG
    junk = os.path.join(tmp_path, "junk.bp")
    with open(junk, "wb") as f:
        f.write(b"not a state file at all" * 10)
    same = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    same.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    with pytest.raises(B.BPError) as e:
        same.load(junk)
    assert e.value.code == B.BP_ERR_IO
    with pytest.raises(B.BPError) as e:
        same.load(os.path.join(tmp_path, "missing.bp"))
    assert e.value.code == B.BP_ERR_IO
    for c in (a, other, same):
        c.close()


def test_async_field_reads_match_synchronous_reads():
    """bp_read_field_async snapshots the field on the device and copies it to
    the host on a side stream while the next steps run (two snapshot buffers
    alternate): each step's E_y, read that way, equals the synchronous read of
    the same step in an identical run."""
    import torch
    wl = small_periodic_3d()
    nsteps = 5
    a, _, _ = gpu_from_workload(wl, deposit_mode=1)
    bufs = [torch.empty(int(np.prod(wl.n)), dtype=torch.float32, pin_memory=True) for _ in range(nsteps)]
    for k in range(nsteps):
        a.step(1)
        a.read_field_async(1, bufs[k].data_ptr())
    a.sync()
    b, _, _ = gpu_from_workload(wl, deposit_mode=1)
    for k in range(nsteps):
        b.step(1)
        b.sync()
        ref = b.read_field(1).ravel()
        assert np.array_equal(bufs[k].numpy(), ref), k
    assert np.abs(bufs[-1].numpy()).max() > 0
    a.close()
    b.close()


def test_state_file_checksum_rejects_truncated_and_corrupted_files(tmp_path):
    """The state file ends with the CRC-32 (zlib's convention) of every byte
    before it.  bp_load checks it before touching the context: a truncated
    file and a file with one flipped bit give BP_ERR_IO, and the context can
    still load the intact file afterwards."""
    import zlib
    from paper_2208_08038_gb300 import binding as B
    wl = small_periodic_3d()
    path = os.path.join(tmp_path, "state.bp")
    a, _, _ = gpu_from_workload(wl, deposit_mode=1)
    a.step(5)
    a.save(path)
    a.sync()
    fa = a.fields()
    data = open(path, "rb").read()
    assert int.from_bytes(data[-4:], "little") == zlib.crc32(data[:-4])
    short = os.path.join(tmp_path, "short.bp")
    open(short, "wb").write(data[: len(data) // 2])
    flipped = bytearray(data)
    flipped[len(data) - 1000] ^= 0x10  # inside the saved fields
    flip = os.path.join(tmp_path, "flip.bp")
    open(flip, "wb").write(bytes(flipped))
    sp = wl.species[0]
    b = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    b.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    for bad in (short, flip):
        with pytest.raises(B.BPError) as e:
            b.load(bad)
        assert e.value.code == B.BP_ERR_IO
    b.load(path)
    b.sync()
    assert np.array_equal(b.fields()[:6], fa[:6])
    a.close()
    b.close()


def test_nonfinite_particles_are_rejected_at_load():
    from paper_2208_08038_gb300 import binding as B
    wl = small_periodic_3d()
    sp = wl.species[0]
    for bad in ("x", "u"):
        ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
        sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
        x, u = sp.x.copy(), sp.u.copy()
        (x if bad == "x" else u)[len(x) // 3, 1] = np.nan
        with pytest.raises(B.BPError) as e:
            ctx.load_particles(sid, x, u)
        assert e.value.code == B.BP_ERR_NONFINITE, bad
        ctx.close()


def _load_pinned(B, ctx, sid, x, u, pidx=None):
    """bp_load_particles from page-locked host arrays (read in place by the
    conversion kernel) instead of the binding's pageable copies (staged)."""
    import torch
    xh = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
    uh = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).pin_memory()
    ph = None if pidx is None else torch.from_numpy(np.ascontiguousarray(pidx, dtype=np.int32)).pin_memory()
    rc = B.lib().bp_load_particles(ctx._h, sid, B._ptr(xh.data_ptr()), B._ptr(uh.data_ptr()),
                                   None if ph is None else B._ptr(ph.data_ptr()), len(x))
    ctx._check(rc, "bp_load_particles")


def test_pinned_and_pageable_loads_give_the_same_state():
    """Both load paths (pinned arrays read in place; pageable arrays staged
    on the device) give the same particles, bit for bit, with and without
    parameter indices, and reject a non-finite position the same way."""
    from paper_2208_08038_gb300 import binding as B
    wl = small_periodic_3d()
    sp = wl.species[0]
    rng = np.random.default_rng(11)
    pidx = rng.integers(0, 1, len(sp.x)).astype(np.int32)
    for idx in (None, pidx):
        out = []
        for pinned in (False, True):
            ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
            sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
            if pinned:
                _load_pinned(B, ctx, sid, sp.x, sp.u, idx)
            else:
                ctx.load_particles(sid, sp.x, sp.u, idx)
            ctx.step(2)
            ctx.sync()
            out.append((np.concatenate(ctx.read_particles(sid, len(sp.x)), axis=1), ctx.fields()))
            ctx.close()
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile)
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    x = sp.x.copy()
    x[len(x) // 2, 0] = np.inf
    with pytest.raises(B.BPError) as e:
        _load_pinned(B, ctx, sid, x, sp.u)
    assert e.value.code == B.BP_ERR_NONFINITE
    ctx.close()


class _BudgetAllocator:
    """A bp_allocator that hands out torch caching-allocator blocks until a
    byte budget is spent, then returns NULL (a caller out of memory)."""

    def __init__(self, budget):
        import ctypes as C
        import torch
        from paper_2208_08038_gb300 import binding as B
        self.left = budget
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, user):
            if nbytes > self.left:
                return None
            self.left -= nbytes
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0))

        def _free(ptr, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a = B.ALLOC_FN(_alloc)
        self._f = B.FREE_FN(_free)
        self.struct = B.Allocator(self._a, self._f, None)


def test_allocator_failure_is_reported_as_oom():
    """An allocator that returns NULL gives BP_ERR_OOM: at creation when it
    fails at once, at the particle load when only the grid fits."""
    from paper_2208_08038_gb300 import binding as B
    wl = small_periodic_3d()
    sp = wl.species[0]
    with pytest.raises(B.BPError) as e:
        B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile, allocator=_BudgetAllocator(0))
    assert e.value.code == B.BP_ERR_OOM
    ncell = int(np.prod(wl.n))
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=1, tile=wl.tile,
                    allocator=_BudgetAllocator(80 * ncell + (1 << 20)))
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    with pytest.raises(B.BPError) as e:
        ctx.load_particles(sid, sp.x, sp.u)
    assert e.value.code == B.BP_ERR_OOM
    ctx.close()
