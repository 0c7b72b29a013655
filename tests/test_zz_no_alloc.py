"""abp_step_static, the allocation-free step, against abp_step_plain.

abp_step_static serves callers that cannot let the bias allocate device
memory inside a step: a plugin whose host MD engine hands out GPU memory from
its own fixed pool, a step loop that a device-wide cudaFree synchronisation
would stall, a long run under a per-process memory limit. It keeps all of its
scratch in one static device array. These tests call it through the C ABI on
two consecutive MD steps (each depositing a hill, so the second call depends
on the first) with a grid the test owns, and check its forces and grid
against the allocating plain form on the same inputs, within the parity
tolerances the other GPU tests use: a 2D COM-distance + dihedral walker in
FP32 and in FP64, and a 3D walker whose third CV is a coordination number
over 40 x 400 atoms, in FP32 and in FP64. The file is collected last, so a
failure here leaves every other test's result standing.
"""
import numpy as np
import pytest

from tests import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(kind):
    from paper_1609_09833_gb300 import synth

    if kind.startswith("mb64"):
        spec = synth.mb64_specs(nw=1, stride=1)[0]  # a hill on every step
        frames = synth.SweepFrames(1, seed=41).frames(0, 2, dtype=np.float64)
    else:
        specs = synth.uneven1000_specs(17, nw=20, stride=1)
        i = next(j for j, s in enumerate(specs) if len(s["grid"]["n"]) == 3)
        spec = specs[i]
        tmpl = synth.uneven1000_templates(17, nw=20)[i]
        frames = synth.JitterFrames([tmpl], seed=43).frames(0, 2, dtype=np.float64)
        assert spec["cvs"][-1]["type"] == "coord"
    return spec, frames


def _grid_fields(grid, d, fp64):
    """[nodes, 1 + d] V_b and its gradient from caller-owned grid records."""
    g = grid.double().cpu().numpy()
    if fp64:
        return g[:, :1 + d]
    c = 2 if d == 1 else 4  # the compensation words follow the values
    return g[:, :1 + d] + g[:, c:c + 1 + d]


@pytest.mark.parametrize("kind", ["mb64_fp32", "mb64_fp64", "cn3d_fp32", "cn3d_fp64"])
def test_static_step_matches_plain_step_on_two_calls(kind):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import abp, build

    build.build()
    abp.load()
    torch.cuda.set_device(0)
    fp64 = kind.endswith("fp64")
    spec, frames = _case(kind)
    natoms = spec["natoms"]
    d = len(spec["grid"]["n"])
    tdt = torch.float64 if fp64 else torch.float32
    cdt = abp.ABP_F64 if fp64 else abp.ABP_F32
    prec = abp.ABP_PREC_FP64 if fp64 else abp.ABP_PREC_FP32_COMP
    rec = abp.to_records(frames, tdt).cuda()
    ctx = abp.Context(0)
    try:
        # the existing entry point: a library-allocated walker, plain form
        walkers = ctx.make_walkers([spec], precision=prec)
        offs = torch.zeros(1, dtype=torch.int64, device="cuda")
        Fp = torch.zeros(2, natoms, 4, dtype=tdt, device="cuda")
        for t in range(2):
            abp.abp_step_plain(ctx.handle, walkers, rec[t], cdt, offs, Fp[t], offs, abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        grid_plain = ctx.bias(walkers[0])

        # the allocation-free entry point: the test owns the (zeroed) grid
        gdesc = abp.grid_desc(spec["grid"], prec)
        nodes = int(np.prod(spec["grid"]["n"]))
        rec_bytes = 16 if d == 1 else 32
        grid = torch.zeros(nodes, rec_bytes // tdt.itemsize, dtype=tdt, device="cuda")
        wdesc, keep = abp.walker_desc(spec)
        Fs = torch.zeros(2, natoms, 4, dtype=tdt, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for t in range(2):
            abp.abp_step_static(0, stream, gdesc, grid, wdesc, rec[t], cdt, Fs[t], abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        del keep
        grid_static = _grid_fields(grid, d, fp64)

        tol_v = 1e-12 if fp64 else P.TOL_V
        tol_f = 1e-10 if fp64 else P.TOL_F
        assert np.all(P.rel_field_err(grid_static, grid_plain) < tol_v)
        # both calls deposited: the hills' support is larger than one stencil box
        nz = np.count_nonzero(grid_static[:, 0])
        assert nz > 0 and np.count_nonzero(grid_plain[:, 0]) == nz
        fp = Fp.cpu().numpy()[..., :3].astype(np.float64)
        fs = Fs.cpu().numpy()[..., :3].astype(np.float64)
        for t in range(2):
            assert P.force_err(fs[t:t + 1], fp[t:t + 1]) < tol_f
        assert np.linalg.norm(fs[1], axis=-1).max() > 0.0
    finally:
        torch.cuda.synchronize()
        ctx.close()


def test_static_step_rejects_walkers_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import abp, build, synth

    build.build()
    abp.load()
    # a coordination number over 10 x 69,990 atoms: its lists and Jacobian need more than 1 MiB
    spec = {"natoms": 70_000,
            "cvs": [{"type": "coord", "a": np.arange(10), "b": np.arange(10, 70_000), "r0": 0.4, "n": 6, "m": 12}],
            "grid": synth.grid((0.0,), (100.0,), (256,), (False,)),
            "hill": synth.hill(0.5, (1.0,), 10, 15.0)}
    gdesc = abp.grid_desc(spec["grid"])
    wdesc, keep = abp.walker_desc(spec)
    dummy = torch.zeros(64, device="cuda")
    with pytest.raises(abp.AbpError) as e:
        abp.abp_step_static(0, None, gdesc, dummy, wdesc, dummy, abp.ABP_F32, dummy, abp.ABP_FORCES_OVERWRITE, 0)
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    assert "ABP_STATIC_SCRATCH_BYTES" in str(e.value)


def test_static_step_reports_rmsd_walkers_as_unsupported():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import abp, build, synth

    build.build()
    abp.load()
    spec = synth.paper_rmsd_specs(nw=1)[0]
    spec = dict(spec, hill=synth.hill(0.5, (0.1, 0.1), 1, 15.0))  # a WT walker, so only the CV is at issue
    gdesc = abp.grid_desc(spec["grid"])
    wdesc, keep = abp.walker_desc(spec)
    dummy = torch.zeros(64, device="cuda")
    with pytest.raises(abp.AbpError) as e:
        abp.abp_step_static(0, None, gdesc, dummy, wdesc, dummy, abp.ABP_F32, dummy, abp.ABP_FORCES_OVERWRITE, 0)
    assert e.value.code == abp.ABP_ERR_UNSUPPORTED
    assert "RMSD" in str(e.value)
