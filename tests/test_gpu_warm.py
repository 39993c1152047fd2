"""Learned warm start: the network kernels against the FP64 reference of
oracle/warm_net.py on the same bfloat16 inputs, training on the GPU, and what
the trained network gains over the flat-film start.

Tolerances: forward outputs are stored in bfloat16 (relative rounding 2^-9)
after float32 accumulation, so |y - y_ref| <= 2^-8 |y_ref| + 1e-3 max|y_ref|;
gradients are float32 sums of exact bfloat16 x float32 products, 1e-4 relative
to their largest entry.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import warm_net as W
from paper_2007_15405_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def bf16_dev(torch, a):
    """bfloat16 device tensor holding exactly bf16_round(a) (set through float32)."""
    r = W.bf16_round(a).astype(np.float32)
    return torch.from_numpy(r.reshape(-1)).cuda().to(torch.bfloat16), r.astype(np.float64)


@pytest.mark.parametrize("cin,cout,dil,relu", [(4, 16, 1, True), (16, 16, 4, True), (16, 1, 1, False),
                                                (3, 5, 2, False)])
def test_conv_forward_and_backward_match_reference(env, cin, cout, dil, relu):
    torch, cfm = env
    L = cfm._lib
    rng = np.random.default_rng(cin * 100 + cout + dil)
    n, nz, ny, nx = 2, 7, 6, 9
    xd, x = bf16_dev(torch, rng.standard_normal((n, cin, nz, ny, nx)))
    wd, w = bf16_dev(torch, rng.standard_normal((cout, cin, 27)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout) * 0.1
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    yd = torch.empty(n * cout * nz * ny * nx, dtype=torch.bfloat16, device="cuda")
    cfm._check(L.cf_conv3d_forward(p(xd), n, cin, nz, ny, nx, p(wd), p(bd), cout, dil, int(relu), p(yd), None))
    y = yd.float().cpu().numpy().reshape(n, cout, nz, ny, nx).astype(np.float64)
    y_ref = W.conv3d(x, w, b.astype(np.float32).astype(np.float64), dil, relu)
    assert (np.abs(y - y_ref) <= 2 ** -8 * np.abs(y_ref) + 1e-3 * np.abs(y_ref).max()).all()

    gy = rng.standard_normal((n, cout, nz, ny, nx)).astype(np.float32)
    gyd = torch.from_numpy(gy.reshape(-1)).cuda()
    gxd = torch.empty(n * cin * nz * ny * nx, dtype=torch.float32, device="cuda")
    gwd = torch.zeros(cout * cin * 27, dtype=torch.float32, device="cuda")
    gbd = torch.zeros(cout, dtype=torch.float32, device="cuda")
    cfm._check(L.cf_conv3d_backward(p(xd), n, cin, nz, ny, nx, p(wd), cout, dil, p(yd), int(relu), p(gyd),
                                    p(gxd), p(gwd), p(gbd), None))
    torch.cuda.synchronize()
    # the reference takes its ReLU mask from the GPU's own (bfloat16) outputs
    gx_ref, gw_ref, gb_ref = W.conv3d_backward(x, w, dil, y, relu, gy.astype(np.float64))
    for got, ref in ((gxd, gx_ref), (gwd, gw_ref), (gbd, gb_ref)):
        g = got.cpu().numpy().reshape(ref.shape).astype(np.float64)
        assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-6


def test_mse_and_adam_match_reference(env):
    torch, cfm = env
    L = cfm._lib
    rng = np.random.default_rng(7)
    m = 1000
    pd_, pr = bf16_dev(torch, rng.standard_normal(m))
    t = rng.standard_normal(m).astype(np.float32)
    mask = (rng.random(m) > 0.4).astype(np.float32)
    td, md = torch.from_numpy(t).cuda(), torch.from_numpy(mask).cuda()
    gd = torch.empty(m, dtype=torch.float32, device="cuda")
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    cfm._check(L.cf_mse(p(pd_), p(td), p(md), m, float(mask.sum()), p(gd), p(ld), None))
    loss_ref, g_ref = W.mse(pr, t, mask)
    assert ld.item() == pytest.approx(loss_ref, rel=1e-5)
    assert np.abs(gd.cpu().numpy() - g_ref).max() <= 1e-6 * np.abs(g_ref).max()
    # three Adam steps with changing gradients
    w = rng.standard_normal(64).astype(np.float32)
    wd = torch.from_numpy(w.copy()).cuda()
    m1 = torch.zeros(64, device="cuda")
    m2 = torch.zeros(64, device="cuda")
    wr, a, v = w.astype(np.float64), np.zeros(64), np.zeros(64)
    for step in range(1, 4):
        g = rng.standard_normal(64).astype(np.float32)
        gdv = torch.from_numpy(g).cuda()
        cfm._check(L.cf_adam(p(wd), None, p(gdv), p(m1), p(m2), 64, 1e-2, 0.9, 0.999, 1e-8, step, None))
        wr, a, v = W.adam(wr, g.astype(np.float64), a, v, step, 1e-2)
    assert np.abs(wd.cpu().numpy() - wr).max() < 1e-6


def test_training_learns_a_known_convolution(env):
    """The network trained with the project's kernels fits a two-channel target
    made by fixed random convolutions of its input: the loss falls by 10x or
    more."""
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    net = warm.WarmNet(seed=1)
    rng = np.random.default_rng(2)
    n, nz, ny, nx = 4, 12, 10, 14
    X = rng.standard_normal((n, 4, nz, ny, nx)).astype(np.float32)
    wt = rng.standard_normal((1, 4, 27)) / np.sqrt(27 * 4)
    wt = np.concatenate([wt, -wt])  # two output channels
    T = W.conv3d(X.astype(np.float64), wt, np.zeros(2), 1, False).astype(np.float32) * 0.5
    M = np.ones_like(T)
    losses = warm.train(net, X, T, M, steps=150, batch=4, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])


def test_fallback_restores_the_flat_film(env):
    """With a velocity limit of zero every start 'misbehaves': the run falls
    back to the flat film, identical to a plain set-up."""
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    wl = I.warm_dataset(1, seed=3)[0]
    net = warm.WarmNet(seed=0)
    sim = cfm.Simulation.from_workload(wl)
    used, _ = warm.warm_start(sim, wl, net, window=5, u_limit=0.0)
    assert not used
    ref = cfm.Simulation.from_workload(wl)
    assert np.array_equal(sim.populations(), ref.populations())


def test_set_densities_reproduces_the_film(env):
    """cf_set_densities with the flat film's own densities gives the state of
    cf_set_film (no jitter): the same populations."""
    torch, cfm = env
    wl = I.warm_dataset(1, seed=4)[0]
    wl.jitter_amp = 0.0
    b = cfm.Simulation.from_workload(wl, set_film=False)
    ref = cfm.Simulation.from_workload(wl)
    f = ref.populations().astype(np.float64)
    rhoA, rhoB = f[0].sum(axis=0), f[1].sum(axis=0)
    b.set_densities(rhoA, rhoB)
    assert np.abs(b.populations() - ref.populations()).max() < 1e-7


@pytest.mark.slow
def test_trained_network_gains_over_the_flat_film(env):
    """Train on equilibria the method generates (24 lattices, 1500 steps),
    then on 4 held-out set-ups the predicted start is closer to equilibrium
    than the flat film, and the warm-started run passes its own residual
    check."""
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    wls = I.warm_dataset(28, seed=11)
    X, T, M = warm.dataset(wls, 1500)
    net = warm.WarmNet(seed=0)
    warm.train(net, X[:24], T[:24], M[:24], steps=300, batch=8, lr=2e-3)
    err_plain, err_warm = [], []
    for k in range(24, 28):
        pred = net.predict(X[k])
        err_plain.append(np.sqrt((T[k] ** 2 * M[k]).sum() / M[k].sum()))
        err_warm.append(np.sqrt(((pred - T[k]) ** 2 * M[k]).sum() / M[k].sum()))
    assert np.mean(err_warm) < 0.7 * np.mean(err_plain), (err_plain, err_warm)
    sim = cfm.Simulation.from_workload(wls[24])
    used, _ = warm.warm_start(sim, wls[24], net)
    assert used


def np_film(phi, wall):
    """The flat film's densities from its phi channel (definition)."""
    ra = np.where(phi > 0.5, I.RHO_MAJ, np.where(phi < -0.5, I.RHO_MIN, I.RHO_MIX)).astype(np.float64)
    rb = np.where(phi > 0.5, I.RHO_MIN, np.where(phi < -0.5, I.RHO_MAJ, I.RHO_MIX)).astype(np.float64)
    if wall:
        ra[0] = rb[0] = 0.0
    return ra, rb


def np_features(sim, wl):
    """The network inputs from their definition, on the host."""
    nz, ny, nx = wl.nz, wl.ny, wl.nx
    ins = sim.cuts()[2].reshape(nz, ny, nx).astype(np.float32)
    z = np.arange(nz, dtype=np.float32)[:, None, None] * np.ones((1, ny, nx), np.float32)
    zm = np.floor(wl.h_top + 0.5)
    phi = np.where(z < zm, 1.0, np.where(z == zm, 0.0, -1.0)).astype(np.float32)
    phi = np.where(ins > 0, -1.0, phi).astype(np.float32)
    if wl.wall:
        phi[0] = 0.0
    lks = np.float32(np.log10(wl.capsules[0].kS) + 2.0)
    x = np.stack([ins, phi, z / np.float32(nz), np.full_like(z, lks)])
    mask = ((ins == 0) & (z >= (1 if wl.wall else 0))).astype(np.float32)
    return x, mask


def test_warm_features_match_their_definition(env):
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    wl = I.warm_dataset(1, seed=21)[0]
    sim = cfm.Simulation.from_workload(wl)
    x, mask = warm.features(sim, wl)
    xr, mr = np_features(sim, wl)
    assert np.array_equal(x, xr) and np.array_equal(mask, mr)


def test_warm_apply_matches_its_definition(env):
    """Film plus corrections on the free fluid (at least 1e-3), film elsewhere,
    each component scaled to the film's mass on the free fluid: the state
    equals cf_set_densities of the same densities made on the host."""
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    wl = I.warm_dataset(1, seed=22)[0]
    a = cfm.Simulation.from_workload(wl, set_film=False)
    x, _ = warm.features(a, wl)
    rng = np.random.default_rng(5)
    d = (0.05 * rng.standard_normal((2,) + x.shape[1:])).astype(np.float32)
    d[0, 3, 5, 7] = -50.0  # clipped at 1e-3
    a.warm_apply(wl.h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, torch.from_numpy(d.reshape(-1)).cuda())
    fa, fb = np_film(x[1], wl.wall)
    free = x[0] == 0
    if wl.wall:
        free[0] = False
    D = I.RHO_MAJ - I.RHO_MIN
    ra = np.where(free, np.maximum(fa + D * d[0].astype(np.float64), 1e-3), fa)
    rb = np.where(free, np.maximum(fb + D * d[1].astype(np.float64), 1e-3), fb)
    for r, f in ((ra, fa), (rb, fb)):
        r[free] *= f[free].sum() / r[free].sum()
    b = cfm.Simulation.from_workload(wl, set_film=False)
    b.set_densities(ra, rb)
    pa, pb = a.populations().astype(np.float64), b.populations().astype(np.float64)
    assert np.abs(pa - pb).max() <= 1e-6 * np.abs(pb).max()


def test_warm_target_matches_its_definition(env):
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    wl = I.warm_dataset(1, seed=23)[0]
    sim = cfm.Simulation.from_workload(wl)
    sim.step(30)
    t = warm.target_of(sim, wl)
    x, mask = np_features(sim, wl)
    fa, fb = np_film(x[1], wl.wall)
    rho, _ = sim.fields()
    D = I.RHO_MAJ - I.RHO_MIN
    ref = np.stack([(rho[0] - fa) / D, (rho[1] - fb) / D]).astype(np.float32) * mask[None]
    assert np.abs(t - ref).max() <= 1e-6


def test_field_check_matches_numpy(env):
    torch, cfm = env
    wl = I.warm_dataset(1, seed=24)[0]
    sim = cfm.Simulation.from_workload(wl)
    sim.step(3)
    c0 = sim.field_check()
    r0, u0 = sim.fields()
    assert c0[0] == 1.0 and c0[1] == r0.min() and c0[2] == np.abs(u0).max()
    assert c0[3] == pytest.approx(np.abs(r0).mean(), rel=1e-12)  # against zero
    sim.step(7)
    c1 = sim.field_check()
    r1, u1 = sim.fields()
    assert c1[1] == r1.min() and c1[2] == np.abs(u1).max()
    assert c1[3] == pytest.approx(np.abs(r1 - r0).mean(), rel=1e-9)


def test_device_warm_start_equals_the_host_construction(env):
    """The prediction made on the device and applied with cf_warm_apply sets
    the state the definition gives for the same network output (read back to
    the host): the prediction is complete before the simulation's stream
    reads it."""
    torch, cfm = env
    from paper_2007_15405_gb300 import warm
    net = warm.WarmNet(seed=3)
    D = I.RHO_MAJ - I.RHO_MIN
    for wl in I.warm_dataset(3, seed=31):
        a = cfm.Simulation.from_workload(wl)
        x, _ = warm.features_dev(a, wl)
        a.warm_apply(wl.h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, net.predict_dev(x, (wl.nz, wl.ny, wl.nx)))
        b = cfm.Simulation.from_workload(wl)
        xh, _ = warm.features(b, wl)
        d = net.predict(xh).astype(np.float64)
        fa, fb = np_film(xh[1], wl.wall)
        free = xh[0] == 0
        if wl.wall:
            free[0] = False
        ra = np.where(free, np.maximum(fa + D * d[0], 1e-3), fa)
        rb = np.where(free, np.maximum(fb + D * d[1], 1e-3), fb)
        for r, f in ((ra, fa), (rb, fb)):
            r[free] *= f[free].sum() / r[free].sum()
        b.set_densities(ra, rb)
        pa, pb = a.populations().astype(np.float64), b.populations().astype(np.float64)
        assert np.abs(pa - pb).max() <= 1e-6 * np.abs(pb).max()
