"""Adjoint gradient (GPU, FP32, checkpointed) against central finite differences of the FP64
oracle: J = x-centroid of fluid 0; parameters = the per-wall-node contact angle theta (triple
(90, 180 - theta, theta)) and the Zou-He inflow velocity.  Finite differences in FP32 would drown
in round-off at h = 1e-3 deg, so they are taken on the FP64 oracle."""
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


def pillar_case():
    """Compound droplet overlapping a pillar, Zou-He inflow, per-node angles in [60, 120].

    The seeded droplet is built from exactly pure nodes (densities exactly 1 and 0); at that
    state the theta-derivative of J is not continuous: any seeded relative perturbation of the
    initial densities (1e-7 or 1e-6, of any one fluid, symmetric or not) moves the FP64 finite
    difference of the largest components by the same 3e-3, and the FP32 trajectory, perturbed by
    its own rounding, follows the perturbed branch.  A 1e-6 seeded perturbation puts both sides
    at a generic point where J is smooth."""
    w = W.pillars(nx=96, ny=48, count=2, r_lo=6.0, r_hi=8.0, x_lo=38.0, x_hi=60.0, gap=6.0,
                  seed=7, drop=(28.0, 24.0), r_core=6.0, r_shell=12.0,
                  theta_range=(60.0, 120.0), u_in=0.02)
    rng = np.random.default_rng(1)
    w.rho = w.rho * (1.0 + 1e-6 * rng.standard_normal(w.rho.shape))
    return w


def flat_case():
    """Janus droplet on a flat wall (periodic x), per-node angle triples jittered around
    (80, 60, 110)."""
    w = W.janus_flat(nx=64, ny=36, R=11.0, triple=(80.0, 60.0, 110.0), sigma=(0.012, 0.009, 0.011))
    rng = np.random.default_rng(3)
    w.angles = w.angles + rng.uniform(-8.0, 8.0, size=w.angles.shape)
    return w


def oracle_J(oracle_mod, w, angles_nodes, idx, u_in, steps, threads=1):
    ang = w.angles.copy().reshape(-1, 3)
    ang[idx] = angles_nodes
    o = oracle_mod.Oracle(w.nx, w.ny, w.periodic_y, w.bc_x, w.solid, ang.reshape(w.angles.shape),
                          w.sigma, w.nu, w.beta0, u_in, w.rho_out, threads=threads)
    o.set_fields(w.rho)
    o.step(steps)
    d = o.diag()
    return d[3] / d[0]


@pytest.mark.parametrize("case", ["pillar", "flat"])
def test_adjoint_matches_fd_of_oracle(gpu, oracle_mod, case):
    import torch
    from paper_2102_04709_gb300 import adjoint

    w = pillar_case() if case == "pillar" else flat_case()
    steps, K = 150, 40          # 4 segments, the last one partial
    sim = gpu.Lbm3.from_workload(w)
    idx = sim.wall_nodes()
    a0 = w.angles.reshape(-1, 3)[idx].copy()
    ang = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    u = torch.tensor(w.u_in, dtype=torch.float64, requires_grad=True)
    J = adjoint.centroid(sim, ang, u, w.rho, steps, K)
    J.backward()
    g_ang = ang.grad.numpy()

    J0 = oracle_J(oracle_mod, w, a0, idx, w.u_in, steps)
    assert abs(J.item() - J0) < 1e-5 * abs(J0)

    # directional derivative along a random direction of all wall-angle triples
    rng = np.random.default_rng(5)
    v = rng.standard_normal(a0.shape)
    h = 1e-3
    fd = (oracle_J(oracle_mod, w, a0 + h * v, idx, w.u_in, steps) -
          oracle_J(oracle_mod, w, a0 - h * v, idx, w.u_in, steps)) / (2 * h)
    ad = float((g_ang * v).sum())
    print(f"{case}: directional dJ/dangles: adjoint {ad:.6e}  fd {fd:.6e}")
    assert abs(fd) > 1e-8, "the wetting must influence J in this case"
    assert abs(ad - fd) <= 1e-3 * abs(fd)

    if w.bc_x == W.BC_ZOUHE:
        hu = 1e-6
        fdu = (oracle_J(oracle_mod, w, a0, idx, w.u_in + hu, steps) -
               oracle_J(oracle_mod, w, a0, idx, w.u_in - hu, steps)) / (2 * hu)
        print(f"{case}: dJ/du: adjoint {u.grad.item():.6e}  fd {fdu:.6e}")
        assert abs(u.grad.item() - fdu) <= 1e-3 * abs(fdu)


def small_case():
    """64 x 32, one pillar wetted by the shell of a compound droplet, Zou-He inflow, per-node
    angles in [60, 120], generic (1e-6 perturbed) initial densities."""
    w = W.pillars(nx=64, ny=32, count=1, r_lo=5.0, r_hi=6.0, x_lo=30.0, x_hi=36.0, gap=4.0,
                  seed=3, drop=(20.0, 16.0), r_core=4.0, r_shell=9.0,
                  theta_range=(60.0, 120.0), u_in=0.02)
    rng = np.random.default_rng(2)
    w.rho = w.rho * (1.0 + 1e-6 * rng.standard_normal(w.rho.shape))
    return w


def _fd_component(job):
    """Central difference of the oracle's J in one wall angle (or in u_in when comp < 0)."""
    from oracle import oracle as om
    w, idx, a0, steps, node, comp, h = job
    if comp < 0:
        jp = oracle_J(om, w, a0, idx, w.u_in + h, steps)
        jm = oracle_J(om, w, a0, idx, w.u_in - h, steps)
    else:
        ap = a0.copy()
        ap[node, comp] += h
        am = a0.copy()
        am[node, comp] -= h
        jp = oracle_J(om, w, ap, idx, w.u_in, steps)
        jm = oracle_J(om, w, am, idx, w.u_in, steps)
    return (jp - jm) / (2 * h)


def test_adjoint_full_gradient_small_case(gpu):
    """Every component of dJ/d(angles) and dJ/du_in on the 64 x 32, 200-step case against a
    central difference of the FP64 oracle per component (a process pool of spawned workers
    runs the 2 (3 n_wall + 1) oracle runs)."""
    import multiprocessing as mp
    import os
    import torch
    from paper_2102_04709_gb300 import adjoint

    w = small_case()
    steps, K = 200, 64
    sim = gpu.Lbm3.from_workload(w)
    idx = sim.wall_nodes()
    a0 = w.angles.reshape(-1, 3)[idx].copy()
    ang = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    u = torch.tensor(w.u_in, dtype=torch.float64, requires_grad=True)
    J = adjoint.centroid(sim, ang, u, w.rho, steps, K)
    J.backward()
    g = ang.grad.numpy()
    jobs = [(w, idx, a0, steps, i, c, 1e-3) for i in range(len(idx)) for c in range(3)]
    jobs.append((w, idx, a0, steps, 0, -1, 1e-6))
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        fd = np.array(pool.map(_fd_component, jobs))
    fd_ang, fd_u = fd[:-1].reshape(-1, 3), fd[-1]
    scale = np.abs(fd_ang).max()
    err = np.abs(g - fd_ang).max()
    print(f"full gradient: {len(idx)} wall nodes, max |dJ/dangle| {scale:.3e}, "
          f"max error {err:.3e}; dJ/du adjoint {u.grad.item():.6e} fd {fd_u:.6e}")
    assert scale > 1e-7
    assert err <= 1e-3 * scale
    assert abs(u.grad.item() - fd_u) <= 1e-3 * abs(fd_u)


@pytest.mark.parametrize("K", [25, 60, 1])
def test_adjoint_leaves_final_state(gpu, K):
    """After lbm3_adjoint_centroid the simulation holds the same state (populations and wall
    values) as after lbm3_step, whether the forward pass kept every state (K = 60), some
    segments (25) or checkpoints only (1)."""
    w = pillar_case()
    a = gpu.Lbm3.from_workload(w)
    a.adjoint_centroid(60, K)
    b = gpu.Lbm3.from_workload(w)
    b.step(60)
    fa, ca = a.get_state()
    fb, cb = b.get_state()
    assert np.array_equal(fa, fb)
    assert np.array_equal(ca, cb)
    a.close()
    b.close()


def test_adjoint_checkpoint_schedules_agree(gpu):
    """The same gradient (to the rounding of the adjoint's atomic sums) with every state kept
    (K = n), with segments recomputed from checkpoints (K = 25, 7, 1), from a second call that
    reuses the device memory the first one kept, and after that memory was released."""
    w = pillar_case()
    n = 60
    sim = gpu.Lbm3.from_workload(w)
    runs = []
    for K in (n, n, 25, 7, 1):
        sim.set_fields(w.rho)
        runs.append(sim.adjoint_centroid(n, K))
    sim.adjoint_release()
    sim.set_fields(w.rho)
    runs.append(sim.adjoint_centroid(n, n))
    J0, g0, u0 = runs[0]
    scale = np.abs(g0).max()
    assert scale > 0
    for J, g, u in runs[1:]:
        assert J == J0
        assert np.abs(g - g0).max() <= 1e-4 * scale
        assert abs(u - u0) <= 1e-5 * abs(u0)
    sim.close()


def test_adjoint_gradients_follow_input_device(gpu):
    """The torch.autograd.Function returns each gradient on its input's device and in its dtype:
    angles and u_in as CUDA tensors give CUDA gradients equal (to the rounding of the adjoint's
    atomic sums) to those of CPU inputs."""
    import torch
    from paper_2102_04709_gb300 import adjoint

    w = pillar_case()
    sim = gpu.Lbm3.from_workload(w)
    idx = sim.wall_nodes()
    a0 = w.angles.reshape(-1, 3)[idx].copy()
    grads = []
    for dev in ("cpu", "cuda"):
        ang = torch.tensor(a0, dtype=torch.float64, device=dev, requires_grad=True)
        u = torch.tensor(w.u_in, dtype=torch.float64, device=dev, requires_grad=True)
        J = adjoint.centroid(sim, ang, u, w.rho, 40, 16)
        (2.0 * J).backward()
        assert ang.grad.device.type == dev and u.grad.device.type == dev
        assert ang.grad.dtype == torch.float64
        grads.append((ang.grad.cpu().numpy(), u.grad.item()))
    # the adjoint kernels scatter with atomic adds, so two runs agree to rounding, not bit for bit
    scale = np.abs(grads[0][0]).max()
    assert np.abs(grads[0][0] - grads[1][0]).max() <= 1e-4 * scale
    assert abs(grads[0][1] - grads[1][1]) <= 1e-6 * abs(grads[0][1])
    sim.close()


def test_adjoint_matches_oracle_reference_tape(gpu, oracle_mod):
    """Every component of dJ/d(angles) and dJ/du_in of the GPU adjoint (FP32, checkpoints every
    64 steps) on the 64 x 32, 200-step case against the oracle's reference tape (the FP64 oracle
    recorded and swept backwards, an independent reverse sweep): within 1e-4 of the largest
    angle component, and dJ/du within 1e-4 relative."""
    import torch
    from paper_2102_04709_gb300 import adjoint

    w = small_case()
    steps = 200
    sim = gpu.Lbm3.from_workload(w)
    idx = sim.wall_nodes()
    a0 = w.angles.reshape(-1, 3)[idx].copy()
    ang = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    u = torch.tensor(w.u_in, dtype=torch.float64, requires_grad=True)
    J = adjoint.centroid(sim, ang, u, w.rho, steps, 64)
    J.backward()
    g = ang.grad.numpy()
    Jt, gt, dut = oracle_mod.tape_centroid_gradient(w, steps)
    gt = gt.reshape(-1, 3)[idx]
    scale = np.abs(gt).max()
    err = np.abs(g - gt).max()
    print(f"tape: J {Jt:.9f} vs GPU {J.item():.9f}; max |dJ/dangle| {scale:.3e}, max |GPU - tape| "
          f"{err:.3e}; dJ/du GPU {u.grad.item():.8e} tape {dut:.8e}")
    assert abs(J.item() - Jt) < 1e-5 * abs(Jt)
    assert scale > 1e-7
    assert err <= 1e-4 * scale
    assert abs(u.grad.item() - dut) <= 1e-4 * abs(dut)


def _c5_J(job):
    """The oracle's J on the 512 x 256 adjoint workload for one perturbed parameter set."""
    from oracle import oracle as om
    w, idx, angles, u_in, steps, threads = job
    return oracle_J(om, w, angles, idx, u_in, steps, threads)


def test_adjoint_config5_against_fd(gpu):
    """The 512 x 256 adjoint workload at its full size and length (six pillars, per-node angles
    in [60, 120], Zou-He inflow 0.01, 2000 steps, checkpoints every 100): the compound droplet's
    shell wets a pillar, so the angle field moves the centroid.  One random directional
    derivative over every wall-angle component (h = 1e-3 deg) and dJ/du (h = 1e-6) of the GPU
    adjoint against central differences of the FP64 oracle, within 1e-3 relative.  The initial
    densities carry a seeded 1e-6 perturbation (a generic point; see pillar_case).  The four
    oracle runs go to a pool of spawned workers, each on a share of the host's cores."""
    import multiprocessing as mp
    import torch
    from oracle import oracle as om
    from paper_2102_04709_gb300 import adjoint

    w = W.config5()
    rng = np.random.default_rng(1)
    w.rho = w.rho * (1.0 + 1e-6 * rng.standard_normal(w.rho.shape))
    sim = gpu.Lbm3.from_workload(w)
    idx = sim.wall_nodes()
    a0 = w.angles.reshape(-1, 3)[idx].copy()
    ang = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    u = torch.tensor(w.u_in, dtype=torch.float64, requires_grad=True)
    J = adjoint.centroid(sim, ang, u, w.rho, w.steps, 100)
    J.backward()
    g = ang.grad.numpy()
    v = np.random.default_rng(5).standard_normal(a0.shape)
    h, hu = 1e-3, 1e-6
    th = max(1, om.host_threads() // 4)
    jobs = [(w, idx, a0 + h * v, w.u_in, w.steps, th), (w, idx, a0 - h * v, w.u_in, w.steps, th),
            (w, idx, a0, w.u_in + hu, w.steps, th), (w, idx, a0, w.u_in - hu, w.steps, th)]
    with mp.get_context("spawn").Pool(4) as pool:
        jp, jm, jup, jum = pool.map(_c5_J, jobs)
    fd = (jp - jm) / (2 * h)
    fdu = (jup - jum) / (2 * hu)
    ad = float((g * v).sum())
    print(f"config5: {len(idx)} wall nodes, |dJ/dangles| {np.linalg.norm(g):.4e}; directional: "
          f"adjoint {ad:.8e} fd {fd:.8e}; dJ/du adjoint {u.grad.item():.8e} fd {fdu:.8e}")
    assert abs(fd) > 1e-7, "the wetting must influence J on this workload"
    assert abs(ad - fd) <= 1e-3 * abs(fd)
    assert abs(u.grad.item() - fdu) <= 1e-3 * abs(fdu)
    sim.close()

