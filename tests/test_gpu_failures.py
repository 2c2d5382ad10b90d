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
