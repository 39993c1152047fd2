"""The allocation-free lattice step (cf_lattice_step_static) against the
context step (cf_step) on a lattice without capsules.

Callers that cannot allocate device memory (a host framework that owns the
device memory as one fixed pool, or code that must not allocate once set-up is
over) get cf_lattice_step_static, which takes its density scratch from a fixed
array inside the library.  Its populations must match what cf_step produces,
for two calls in a row (the second call reuses the scratch left by the first).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the parity tolerance of the population comparisons


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_15405_gb300 import build
    build.build()
    from paper_2007_15405_gb300 import capfilm
    capfilm.load_library()
    return torch, capfilm


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("wall,tau", [(1, (1.0, 1.0)), (0, (1.0, 1.0)), (1, (0.8, 1.3))])
def test_static_scratch_step_matches_context_step(env, wall, tau):
    """tau = (1, 1) stores the equilibria; (0.8, 1.3) also relaxes the pulled
    populations and weights the common velocity by 1/tau, so both terms of
    the BGK step are compared."""
    torch, cfm = env
    wl = I.Workload("static", 45, 14, 12, h_top=5.5, capsules=[], steps=2, wall=wall, seed=21,
                    tau=tau)
    sim = cfm.Simulation.from_workload(wl)
    f0 = sim.populations()
    sim.step(1)
    f1 = sim.populations()
    sim.step(1)
    f2 = sim.populations()
    sim.close()

    stream = torch.cuda.current_stream()
    a = torch.from_numpy(f0).cuda()
    # the substrate plane z = 0 of the output is never written: start it from
    # zeros like the context's own buffers, and compare the fluid planes
    b = torch.zeros_like(a)
    # two calls in a row through the C ABI, device buffers owned by the caller
    cfm.lattice_step_static(a.data_ptr(), b.data_ptr(), wl.nx, wl.ny, wl.nz, wall, wl.tau, wl.G,
                            stream.cuda_stream)
    cfm.lattice_step_static(b.data_ptr(), a.data_ptr(), wl.nx, wl.ny, wl.nz, wall, wl.tau, wl.G,
                            stream.cuda_stream)
    torch.cuda.synchronize()
    z0 = 1 if wall else 0
    g1 = b.cpu().numpy().astype(np.float64)[:, :, z0:]
    g2 = a.cpu().numpy().astype(np.float64)[:, :, z0:]
    assert rel(g1, f1.astype(np.float64)[:, :, z0:]) < TOL
    assert rel(g2, f2.astype(np.float64)[:, :, z0:]) < TOL


def test_static_scratch_rejects_oversized_lattice(env):
    torch, cfm = env
    a = torch.zeros(38 * 27, device="cuda")
    with pytest.raises(cfm.CapfilmError, match="static scratch"):
        cfm.lattice_step_static(a.data_ptr(), a.data_ptr(), 1024, 1024, 3, 1, (1.0, 1.0), 3.6)


def test_static_scratch_more_planes_than_a_grid_holds(env):
    """3 x 3 x 116508 = 1048572 nodes fits the scratch but has more fluid
    planes than a launch grid holds in z (65535): the passes stride over the
    planes, so every plane is stepped.  A uniform rest state with G = 0 is a
    fixed point, so each fluid plane must come out equal to its input."""
    torch, cfm = env
    nx, ny, nz = 3, 3, 116508
    w = torch.tensor([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=torch.float32, device="cuda")
    a = torch.empty(2, 19, nz, ny, nx, device="cuda")
    a[0] = (w * 0.6)[:, None, None, None]
    a[1] = (w * 0.2)[:, None, None, None]
    a[:, :, 0] = 0.0
    b = torch.zeros_like(a)
    cfm.lattice_step_static(a.data_ptr(), b.data_ptr(), nx, ny, nz, 1, (1.0, 1.0), 0.0)
    torch.cuda.synchronize()
    d = (b[:, :, 1:] - a[:, :, 1:]).abs().max().item()
    assert d < 1e-7, d


def test_static_scratch_rejects_overlapping_buffers(env):
    """In place (src == dst) the collide pass would overwrite populations its
    neighbours still read: rejected."""
    torch, cfm = env
    n = 2 * 19 * 8 * 8 * 8
    a = torch.zeros(2 * n, device="cuda")
    with pytest.raises(cfm.CapfilmError, match="overlap"):
        cfm.lattice_step_static(a.data_ptr(), a.data_ptr(), 8, 8, 8, 1, (1.0, 1.0), 3.6)
    with pytest.raises(cfm.CapfilmError, match="overlap"):
        cfm.lattice_step_static(a.data_ptr(), a.data_ptr() + 4 * (n // 2), 8, 8, 8, 1, (1.0, 1.0), 3.6)
    # adjacent, non-overlapping halves are accepted
    cfm.lattice_step_static(a.data_ptr(), a.data_ptr() + 4 * n, 8, 8, 8, 1, (1.0, 1.0), 3.6)
    torch.cuda.synchronize()
