"""lbm3_diag_fields, the allocation-free diagnostics entry point, against lbm3_diag on the same
state.  Both accumulate in FP64 the FP32 per-node densities, so sums agree to FP64 rounding of
a different summation order (relative 1e-9 here); max |u| reads the same FP32 velocity and
agrees exactly.  Collected last so that it runs after every other GPU test as well as alone."""
import numpy as np
import pytest

from paper_2102_04709_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_04709_gb300 import build, lbm3
    build.build()
    lbm3.load()
    return lbm3


def call(gpu, torch, sim, w, solid, out):
    rho, u = sim.fields()
    r = torch.tensor(rho, dtype=torch.float32, device="cuda")
    v = torch.tensor(u, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    gpu.diag_fields(r.data_ptr(), v.data_ptr(), solid.data_ptr(), w.nx, w.ny, out.data_ptr())
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return out.cpu().numpy(), free1 - free0


def check(got, ref):
    assert np.allclose(got[:5], ref[:5], rtol=1e-9, atol=0)
    assert got[5] == ref[5]
    assert np.isclose(got[6], ref[6], rtol=1e-9, atol=0)
    assert got[7] == ref[7] == 0


def test_diag_fields_matches_diag_on_consecutive_calls(gpu):
    import torch
    w = W.janus_cylinder(nx=96, ny=90, Rs=16.0, Rj=14.0)
    sim = gpu.Lbm3.from_workload(w)
    solid = torch.tensor(w.solid, dtype=torch.uint8, device="cuda")
    outs = [torch.full((8,), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
    sim.step(40)
    ref = sim.diag()
    a, _ = call(gpu, torch, sim, w, solid, outs[0])
    b, dfree = call(gpu, torch, sim, w, solid, outs[1])
    check(a, ref)
    check(b, ref)
    assert np.array_equal(a, b)
    assert dfree == 0, "the call changed the device's free memory"
    # a later state through the same fixed scratch
    sim.step(25)
    ref2 = sim.diag()
    c, dfree = call(gpu, torch, sim, w, solid, outs[0])
    check(c, ref2)
    assert dfree == 0


def test_diag_fields_large_grid_and_bad_arguments(gpu):
    """A grid spanning the full block count (ragged last block) and the argument checks."""
    import torch
    nx, ny = 1531, 1207                       # 1,847,917 nodes: 1024 blocks, 7 nodes per thread
    g = torch.Generator(device="cpu").manual_seed(4)
    rho = torch.rand((3, ny, nx), generator=g, dtype=torch.float32)
    u = (torch.rand((2, ny, nx), generator=g, dtype=torch.float32) - 0.5) * 0.1
    solid = (torch.rand((ny, nx), generator=g) < 0.2).to(torch.uint8)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    rd, ud, sd = rho.cuda(), u.cuda(), solid.cuda()
    gpu.diag_fields(rd.data_ptr(), ud.data_ptr(), sd.data_ptr(), nx, ny, out.data_ptr())
    got = out.cpu().numpy()
    # expected values from float64 numpy on the host
    r = rho.double().numpy()
    f = solid.numpy() == 0
    yy, xx = np.mgrid[0:ny, 0:nx]
    exp = [r[0][f].sum(), r[1][f].sum(), r[2][f].sum(), (xx * r[0])[f].sum(), (yy * r[0])[f].sum(),
           np.sqrt((u.double().numpy() ** 2).sum(0))[f].max(), r.sum(0)[f].min(), 0.0]
    assert np.allclose(got, exp, rtol=1e-12, atol=0)
    with pytest.raises(gpu.Lbm3Error) as e:
        gpu.diag_fields(rd.data_ptr(), ud.data_ptr(), sd.data_ptr(), 65536, 65536, out.data_ptr())
    assert e.value.code == gpu.LBM3_ERR_TOO_LARGE
    with pytest.raises(gpu.Lbm3Error) as e:
        gpu.diag_fields(0, ud.data_ptr(), sd.data_ptr(), nx, ny, out.data_ptr())
    assert e.value.code == gpu.LBM3_ERR_INVALID
