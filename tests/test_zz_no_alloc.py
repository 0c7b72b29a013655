"""abp_step_static, the allocation-free step, against abp_step_plain.

Some callers cannot call cudaMalloc: a host routine that runs while a CUDA
graph is being captured, a plugin confined to another program's memory pool,
a bias call made where the device allocator must not be touched. For them
abp_step_static keeps all of its scratch in one static device array. This
test calls it through the C ABI on two consecutive MD steps (each depositing
a hill, so the second call depends on the first) with a grid the test owns,
and checks its forces and grid against the allocating plain form on the same
inputs, within the parity tolerances the other GPU tests use. The file is
collected last, so a failure here leaves every other test's result standing.
"""
import numpy as np
import pytest

from tests import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_step_matches_plain_step_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import abp, build, synth

    build.build()
    abp.load()
    torch.cuda.set_device(0)
    spec = synth.mb64_specs(nw=1, stride=1)[0]  # a hill on every step
    natoms = spec["natoms"]
    frames = synth.SweepFrames(1, seed=41).frames(0, 2)
    rec = abp.to_records(frames).cuda()
    ctx = abp.Context(0)
    try:
        # the existing entry point: a library-allocated walker, plain form
        walkers = ctx.make_walkers([spec])
        offs = torch.zeros(1, dtype=torch.int64, device="cuda")
        Fp = torch.zeros(2, natoms, 4, device="cuda")
        for t in range(2):
            abp.abp_step_plain(ctx.handle, walkers, rec[t], abp.ABP_F32, offs, Fp[t], offs,
                               abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        grid_plain = ctx.bias(walkers[0])

        # the allocation-free entry point: the test owns the (zeroed) grid
        gdesc = abp.grid_desc(spec["grid"])
        nodes = int(np.prod(spec["grid"]["n"]))
        grid = torch.zeros(nodes, 8, dtype=torch.float32, device="cuda")  # 32-byte records
        wdesc, keep = abp.walker_desc(spec)
        Fs = torch.zeros(2, natoms, 4, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for t in range(2):
            abp.abp_step_static(0, stream, gdesc, grid, wdesc, rec[t], abp.ABP_F32, Fs[t],
                                abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        del keep
        g = grid.double().cpu().numpy()
        grid_static = g[:, 0:3] + g[:, 4:7]  # value + compensation of V, dV0, dV1

        assert np.all(P.rel_field_err(grid_static, grid_plain) < P.TOL_V)
        # both calls deposited: the support exceeds one 47 x 35 stencil box
        assert np.count_nonzero(grid_static[:, 0]) > 47 * 35
        fp = Fp.cpu().numpy()[..., :3].astype(np.float64)
        fs = Fs.cpu().numpy()[..., :3].astype(np.float64)
        for t in range(2):
            assert P.force_err(fs[t:t + 1], fp[t:t + 1]) < P.TOL_F
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
