"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances: relative field L2 <= 1e-5 after one
step and <= 1e-3 at the end of a run (FP32 against FP64); sorted-deposit
reruns bit-identical."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth
from _common import field_rel_l2, gpu_from_workload, oracle_from_workload, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2208_08038_gb300 import binding
    binding.lib()


def run_both(wl, steps, mode=1, check_steps=(), tile=None):
    ora, osid, opid = oracle_from_workload(wl, probe_cap=steps)
    gpu, gsid, gpid = gpu_from_workload(wl, deposit_mode=mode, tile=tile, probe_cap=steps)
    out = []
    done = 0
    for s in sorted(set(check_steps) | {steps}):
        ora.step(s - done)
        gpu.step(s - done)
        gpu.sync()
        done = s
        out.append((s, field_rel_l2(gpu.fields(), ora.fields()), rel_l2(gpu.fields()[6:9], ora.fields()[6:9])))
    return ora, gpu, osid, gsid, opid, gpid, out


# ---------------------------------------------------------------------------
# Yee only

@pytest.mark.parametrize("D", [1, 2, 3])
def test_vacuum_yee_parity(D):
    n = [64, 32, 16][:D]
    dx = [0.2, 0.25, 0.3][:D]
    dt = 0.9 / math.sqrt(sum(1 / d ** 2 for d in dx))
    bc = [1] + [0] * (D - 1)
    wl = synth.Workload("vac", D, tuple(n), tuple(dx), dt, tuple(bc), 40, [], [], tile=(0, 0, 0)[:D])
    ora, _, _ = oracle_from_workload(wl)
    gpu, _, _ = gpu_from_workload(wl)
    rng = np.random.default_rng(D)
    for c in range(6):
        f = rng.normal(size=ora.field(c).shape)
        ora.field(c)[...] = f
        gpu.write_field(c, f.astype(np.float32))
    ora.field(0)[...] = gpu.read_field(0)  # identical FP32-representable start
    for c in range(6):
        ora.field(c)[...] = gpu.read_field(c)
    ora.step(1)
    gpu.step(1)
    gpu.sync()
    assert field_rel_l2(gpu.fields(), ora.fields()) < 1e-6
    ora.step(39)
    gpu.step(39)
    gpu.sync()
    assert field_rel_l2(gpu.fields(), ora.fields()) < 1e-5


# ---------------------------------------------------------------------------
# the 1D neutral medium (2048 cells)

def test_neutral_1d_one_step_and_short_run():
    wl = synth.neutral_1d(ppc=16, steps=400)
    ora, gpu, osid, gsid, opid, gpid, out = run_both(wl, 400, check_steps=(1,))
    (s1, f1, j1), (s2, f2, j2) = out
    assert f1 < 1e-5, out
    assert f2 < 1e-3, out
    x1o, x2o, u1o, u2o = ora.bodies(osid[0])
    x1g, x2g, u1g, u2g = gpu.read_particles(gsid[0], len(x1o))
    assert rel_l2(x1g[:, 0] - x2g[:, 0], x1o[:, 0] - x2o[:, 0]) < 1e-3 or np.abs(x1o - x2o).max() < 1e-12
    assert rel_l2(u2g, u2o) < 1e-3
    assert rel_l2(gpu.read_probe(gpid), ora.probe(opid, 1)) < 1e-3


@pytest.mark.slow
def test_neutral_1d_full_run():
    """The 1D neutral medium at full size and length (16 ions/cell, 3000 steps): relative
    field L2 <= 1e-5 after one step and <= 1e-3 at the end; probe trace too."""
    wl = synth.neutral_1d()
    ora, gpu, osid, gsid, opid, gpid, out = run_both(wl, wl.steps, check_steps=(1,))
    assert out[0][1] < 1e-5, out
    assert out[-1][1] < 1e-3, out
    assert rel_l2(gpu.read_probe(gpid), ora.probe(opid, 1)) < 1e-3


# ---------------------------------------------------------------------------
# 3D thermal medium, several tiles, ragged occupancy, re-sorting

def small_3d(sigma=2e-2, seed=2, steps=30, n=(48, 16, 16), periodic=False):
    wl = synth.neutral_3d(seed=seed, steps=steps, n=n, ppc=4, sigma_u=sigma, margin=3)
    wl.lasers[0].waist = 0.5 * synth.LAMBDA0
    if periodic:  # fast ions would otherwise leave through the open x faces
        wl.bc = (0, 0, 0)
    return wl


def test_written_field_reaches_the_push():
    """The push stages no field box whose neighbouring tiles never held a
    non-zero E or B.  A field written from outside the step (here a local E_y
    blob in a medium that has seen no field) re-marks the tiles, so the ions
    under it are kicked and deposit exactly as in the oracle; the rest of the
    medium stays quiet."""
    wl = small_3d(periodic=True)
    wl.lasers = []
    ora, osid, _ = oracle_from_workload(wl)
    gpu, gsid, _ = gpu_from_workload(wl)
    ora.step(1)
    gpu.step(1)
    gpu.sync()
    assert np.abs(gpu.fields()[:6]).max() == 0.0
    f = np.zeros(ora.field(1).shape, dtype=np.float32)
    f[5:11, 4:9, 30:37] = 2e-3  # [z][y][x]: x cells 30..36; the tiles of x cells 0..15 stay unmarked
    gpu.write_field(1, f)
    ora.field(1)[...] = f
    for _ in range(3):
        ora.step(1)
        gpu.step(1)
    gpu.sync()
    assert field_rel_l2(gpu.fields(), ora.fields()) < 1e-5
    assert rel_l2(gpu.fields()[7], ora.fields()[7]) < 1e-4  # J_y of the kicked ions
    x1o, x2o, u1o, u2o = ora.bodies(osid[0])
    x1g, x2g, u1g, u2g = gpu.read_particles(gsid[0], len(x1o))
    assert np.abs(u2o).max() > 0 and rel_l2(u2g, u2o) < 1e-5
    gpu.close()
    ora.close()


def test_record_capacity_does_not_change_the_fields():
    """Sorted mode: a particle whose nearest node changes in a step leaves a
    five-node record that a separate kernel adds to the fixed-point current,
    or deposits in place when the record buffer is full.  Both add the same
    integers, so with room for a single record (nearly every such particle
    deposited in place) the fields are bit-identical to the default."""
    wl = small_3d(sigma=0.2, periodic=True)  # hot ions: many nearest-node changes per step
    outs = []
    for cap in (0, 1):
        gpu, _, _ = gpu_from_workload(wl)
        if cap:
            gpu.set_record_capacity(cap)
        gpu.step(10)
        gpu.sync()
        outs.append(gpu.fields())
        gpu.close()
    assert np.abs(outs[0][6:9]).max() > 0
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("mode", [0, 1])
def test_3d_thermal_parity(mode):
    wl = small_3d()
    ora, gpu, osid, gsid, opid, gpid, out = run_both(wl, 30, mode=mode, check_steps=(1,))
    assert out[0][1] < 1e-5 and out[0][2] < 1e-4, out
    assert out[-1][1] < 1e-3 and out[-1][2] < 1e-3, out
    x1o, x2o, u1o, u2o = ora.bodies(osid[0])
    x1g, x2g, u1g, u2g = gpu.read_particles(gsid[0], len(x1o))
    L = np.array(wl.n) * np.array(wl.dx)
    d = (x1g - x1o + 0.5 * L) % L - 0.5 * L
    assert np.abs(d).max() < 1e-5
    assert rel_l2(u1g, u1o) < 1e-5


def test_3d_resort_path():
    """Fast thermal ions cross tile margins: the device-triggered re-sort runs
    and the fields still track the oracle."""
    wl = small_3d(sigma=0.15, steps=40, periodic=True)
    ora, gpu, osid, gsid, opid, gpid, out = run_both(wl, 40, check_steps=(1, 20))
    assert out[0][1] < 1e-5, out
    assert all(o[1] < 1e-3 for o in out), out
    n_o = ora.species_info(osid[0])["n"]
    x1g, _, _, _ = gpu.read_particles(gsid[0], n_o)
    assert len(x1g) == n_o


def test_sorted_mode_bit_exact_rerun():
    wl = small_3d(sigma=0.1, steps=25, periodic=True)
    res = []
    for _ in range(2):
        gpu, _, _ = gpu_from_workload(wl, deposit_mode=1)
        gpu.step(25)
        gpu.sync()
        res.append(gpu.fields())
        gpu.close()
    assert np.array_equal(res[0], res[1])


def test_atomic_matches_sorted():
    wl = small_3d(sigma=0.05, steps=10, periodic=True)
    out = []
    for mode in (0, 1):
        gpu, _, _ = gpu_from_workload(wl, deposit_mode=mode)
        gpu.step(10)
        gpu.sync()
        out.append(gpu.fields())
        gpu.close()
    assert field_rel_l2(out[0], out[1], comps=range(9)) < 1e-5


def test_gauss_residual_conserved_gpu():
    """div E - rho (FP64 on the GPU from the FP32 state) keeps its initial
    value up to FP32 rounding of positions: the deposit is charge conserving.
    Scale: the charge density q w of a single body."""
    wl = small_3d(sigma=0.05, steps=20, periodic=True)
    wl.lasers = []
    gpu, _, _ = gpu_from_workload(wl)
    R0 = gpu.residual()
    gpu.step(20)
    gpu.sync()
    R = gpu.residual()
    qw = abs(wl.species[0].w)
    assert np.abs(R - R0).max() < 1e-4 * qw


# ---------------------------------------------------------------------------
# 2D: reduced Bragg crystal; charged ions with free electrons

def test_2d_bragg_small_parity():
    wl = synth.bragg_2d(seed=1, n=256, cells_per_lambda=16, sites=(6, 6), waist_lambda=3.0,
                             fwhm_lambda=3.0, nb=0.05, steps=300)
    ora, gpu, *_ , out = run_both(wl, 300, check_steps=(1,))
    assert out[0][1] < 1e-5, out
    assert out[-1][1] < 1e-3, out


def test_2d_free_electrons_and_charged_ions():
    wl = synth.ionized_crystal_2d(n=(256, 64), span=(2.0, 6.0), steps=60, a0=0.3)
    wl.lasers[0].fwhm = 2 * synth.T0
    wl.lasers[0].t0 = 1.5 * wl.lasers[0].fwhm
    ora, gpu, osid, gsid, opid, gpid, out = run_both(wl, 60, check_steps=(1,))
    assert out[0][1] < 1e-5, out
    assert out[-1][1] < 1e-3, out


def test_empty_species_and_vacuum_laser():
    wl = synth.neutral_1d(ppc=1, steps=200, vacuum=True)
    wl.species = [synth.TwoBody(Zb=1.0, qc=0.0, mc=synth.M_AU, w=0.01, lambda0_m=12.4e-9,
                                omega_b=np.array([3.0]), x=np.zeros((0, 1)), u=np.zeros((0, 3)))]
    ora, gpu, *_ , out = run_both(wl, 200, check_steps=(1,))
    assert out[0][1] < 1e-5 and out[-1][1] < 1e-4, out


def test_errors_are_status_codes():
    from paper_2208_08038_gb300 import binding as B
    with pytest.raises(B.BPError) as e:
        B.Context(1, (64,), (0.1,), 0.2, (1,))
    assert e.value.code == B.BP_ERR_CFL
    with pytest.raises(B.BPError) as e:
        B.Context(2, (60, 64), (0.1, 0.1), 0.05, (1, 0))  # 60 is not a multiple of the 16-cell tile
    assert e.value.code == B.BP_ERR_ARG
    with pytest.raises(B.BPError) as e:
        B.Context(1, (64,), (0.1,), 0.09, (1,), tile=(32,))  # tiles are fixed per dimension
    assert e.value.code == B.BP_ERR_ARG
    ctx = B.Context(1, (64,), (0.1,), 0.09, (1,))
    with pytest.raises(B.BPError) as e:
        ctx.add_two_body(1.0, 0.0, synth.M_AU, 0.01, 12.4e-9, [30.0])  # omega_b dt >= 2
    assert e.value.code == B.BP_ERR_CFL
    sid = ctx.add_two_body(1.0, 0.0, synth.M_AU, 0.01, 12.4e-9, [3.0])
    with pytest.raises(B.BPError) as e:
        ctx.load_particles(sid, np.array([[100.0]]))  # outside the open grid
    assert e.value.code == B.BP_ERR_DOMAIN
