"""Failure detection on the GPU, with every failure made on the host: a state with a non-finite
or a negative population is loaded through lbm3_set_state, and lbm3_diag must report it as
LBM3_ERR_DIVERGED with the offending counts; afterwards a clean state runs on in the same context.
A step before lbm3_set_fields is refused with LBM3_ERR_STATE."""
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


def fluid_node(w):
    """A fluid node in the middle of the droplet (away from walls)."""
    ys, xs = np.nonzero(w.rho[0] > 0.5)
    j = len(xs) // 2
    return ys[j], xs[j]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp16"])
def test_non_finite_population_is_reported_and_recoverable(gpu, precision):
    w = W.janus_flat(nx=96, ny=48, R=14.0)
    sim = gpu.Lbm3.from_workload(w, precision=precision)
    sim.step(20)
    f, c = sim.get_state()
    y, x = fluid_node(w)
    bad = f.copy()
    bad[0, 3, y, x] = np.nan
    sim.set_state(bad, c)
    sim.step(2)
    with pytest.raises(gpu.Lbm3Error) as e:
        sim.diag()
    assert e.value.code == gpu.LBM3_ERR_DIVERGED
    d = sim.diag(check=False)
    assert d[7] > 0 and np.isnan(d[0])
    # the context is still usable: a clean state steps and checks out
    sim.set_state(f, c)
    sim.step(5)
    d = sim.diag()
    assert d[7] == 0 and np.isfinite(d[:3]).all()
    sim.close()


def test_non_positive_density_is_reported(gpu):
    w = W.janus_flat(nx=96, ny=48, R=14.0)
    sim = gpu.Lbm3.from_workload(w)
    f, c = sim.get_state()
    y, x = fluid_node(w)
    f[:, :, y - 1:y + 2, x - 1:x + 2] = -0.01  # the node pulls only negative populations
    sim.set_state(f, c)
    with pytest.raises(gpu.Lbm3Error) as e:
        sim.diag()
    assert e.value.code == gpu.LBM3_ERR_DIVERGED
    d = sim.diag(check=False)
    assert d[6] <= 0 and d[7] == 0
    sim.close()


def test_step_before_fields_is_refused(gpu):
    w = W.janus_flat(nx=64, ny=32, R=10.0)
    sim = gpu.Lbm3.from_workload(w, init=False)
    for call in (lambda: sim.step(1), sim.diag, sim.fields):
        with pytest.raises(gpu.Lbm3Error) as e:
            call()
        assert e.value.code == gpu.LBM3_ERR_STATE
    sim.set_fields(w.rho)
    sim.step(1)
    assert sim.diag()[7] == 0
    sim.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp16"])
def test_copy_wait_timeout_is_reported_once_and_recoverable(gpu, precision):
    """The bounded wait of the bulk-copy step kernels, made to run out: with a wait limit of 0
    polls every block of the pure-tile kernel gives up at its first tile, sets the error bit,
    drains the copies it issued (full limit) and returns.  lbm3_diag then reports LBM3_ERR_CUDA
    once; after a clean lbm3_set_state and the default limit the run steps on and matches an
    untouched run bit for bit.  Nothing faults or hangs: the drained copies have completed
    before each block exits, and the skipped tiles only leave old values in the output buffer."""
    w = W.pillars(nx=200, ny=96, count=3, r_lo=8.0, r_hi=12.0, x_lo=90.0, x_hi=180.0, gap=6.0,
                  seed=5, drop=(50.0, 48.0), r_core=10.0, r_shell=18.0, u_in=0.02)
    assert w.nx % 8 == 0
    sim = gpu.Lbm3.from_workload(w, precision=precision)
    assert sim.info()["tma"], "the bulk-copy path must be active for this test"
    sim.step(10)
    f, c = sim.get_state()
    sim.set_copy_wait_limit(0)
    sim.step(3)
    with pytest.raises(gpu.Lbm3Error) as e:
        sim.diag()
    assert e.value.code == gpu.LBM3_ERR_CUDA and "bulk tensor copy" in str(e.value)
    sim.diag(check=False)                      # reported once, then cleared
    sim.set_copy_wait_limit(-1)
    sim.set_state(f, c)
    sim.step(20)
    sim.diag()
    ref = gpu.Lbm3.from_workload(w, precision=precision)
    ref.step(10)
    ref.set_state(*ref.get_state())
    ref.step(20)
    assert np.array_equal(sim.fields()[0], ref.fields()[0])
    # the error bit also reaches lbm3_fields
    sim.set_copy_wait_limit(0)
    sim.step(1)
    with pytest.raises(gpu.Lbm3Error) as e:
        sim.fields()
    assert e.value.code == gpu.LBM3_ERR_CUDA
    sim.close()
    ref.close()
