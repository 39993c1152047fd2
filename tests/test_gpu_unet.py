"""The tensor-core U-net layers (cf_unet_*) against the FP64 definitions of
oracle/warm_net.py, on identical bfloat16 inputs (values rounded to bfloat16
first, so both sides multiply the same numbers).

Tolerances: float outputs of a convolution accumulate exact bf16 products in
float32, so they agree with FP64 to ~1e-6 of the output scale (5e-6 asserted);
bfloat16 outputs add one rounding (2^-8 relative).  Layout changes, pooling,
upsampling and concatenation are exact (or one bf16 rounding of a mean)."""
import numpy as np
import pytest

from oracle import warm_net as W

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


def bf16_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def p(t):
    return t.data_ptr() if t is not None else None


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SHAPES = [(1, 4, 6, 8, 16, 8), (2, 5, 3, 7, 32, 40), (1, 6, 6, 6, 48, 16)]


@pytest.mark.parametrize("n,nz,ny,nx,cin,cout", SHAPES)
def test_conv_forward(env, n, nz, ny, nx, cin, cout):
    torch, cfm = env
    L = cfm.load_library()
    rng = np.random.default_rng(cin + cout)
    x = W.bf16_round(rng.standard_normal((n, nz, ny, nx, cin)))
    w = W.bf16_round(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    ref = W.conv3d_cl(x, w, b.astype(np.float64), False)
    xd, wd = bf16_dev(torch, x), bf16_dev(torch, w)
    bd = torch.from_numpy(b).cuda()
    yf = torch.empty(n * nz * ny * nx * cout, device="cuda")
    cfm._check(L.cf_unet_conv(p(xd), n, nz, ny, nx, cin, p(wd), p(bd), cout, 0, 1, p(yf), None))
    yb = torch.empty(n * nz * ny * nx * cout, device="cuda", dtype=torch.bfloat16)
    cfm._check(L.cf_unet_conv(p(xd), n, nz, ny, nx, cin, p(wd), p(bd), cout, 1, 0, p(yb), None))
    torch.cuda.synchronize()
    got = host(yf).reshape(ref.shape)
    assert rel(got, ref) < 5e-6
    gotb = host(yb).reshape(ref.shape)
    assert np.abs(gotb - np.maximum(ref, 0)).max() <= 2 ** -8 * np.abs(ref).max() + 1e-7


TC_SHAPES = [(1, 4, 6, 8, 16, 16), (2, 5, 3, 7, 32, 48), (1, 6, 6, 6, 48, 16), (3, 4, 4, 8, 32, 32),
             (1, 8, 10, 12, 192, 64), (1, 4, 8, 16, 128, 128), (1, 8, 8, 8, 32, 16)]


@pytest.mark.parametrize("n,nz,ny,nx,cin,cout", TC_SHAPES)
def test_conv_tensor_memory_path(env, n, nz, ny, nx, cin, cout):
    """cf_unet_conv_tc (tcgen05 MMAs, accumulators in tensor memory) against
    the FP64 definition, over tiles of 128 voxels with ragged tails, across
    samples of a batch, and for every channel count the network uses."""
    torch, cfm = env
    L = cfm.load_library()
    rng = np.random.default_rng(7 * cin + cout + n)
    x = W.bf16_round(rng.standard_normal((n, nz, ny, nx, cin)))
    w = W.bf16_round(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    ref = W.conv3d_cl(x, w, b.astype(np.float64), False)
    xd, wd = bf16_dev(torch, x), bf16_dev(torch, w)
    bd = torch.from_numpy(b).cuda()
    yf = torch.empty(n * nz * ny * nx * cout, device="cuda")
    cfm._check(L.cf_unet_conv_tc(p(xd), n, nz, ny, nx, cin, p(wd), p(bd), cout, 0, 1, p(yf), None))
    yb = torch.empty(n * nz * ny * nx * cout, device="cuda", dtype=torch.bfloat16)
    cfm._check(L.cf_unet_conv_tc(p(xd), n, nz, ny, nx, cin, p(wd), p(bd), cout, 1, 0, p(yb), None))
    import ctypes
    err = ctypes.c_uint(7)
    cfm._check(L.cf_unet_tc_error(ctypes.byref(err)))
    assert err.value == 0
    got = host(yf).reshape(ref.shape)
    assert rel(got, ref) < 5e-6, rel(got, ref)
    gotb = host(yb).reshape(ref.shape)
    assert np.abs(gotb - np.maximum(ref, 0)).max() <= 2 ** -8 * np.abs(ref).max() + 1e-7


def test_conv_tensor_memory_path_rejects_bad_shapes(env):
    torch, cfm = env
    L = cfm.load_library()
    x = torch.zeros(4 * 4 * 4 * 16, device="cuda", dtype=torch.bfloat16)
    w = torch.zeros(27 * 8 * 16, device="cuda", dtype=torch.bfloat16)
    y = torch.zeros(4 * 4 * 4 * 8, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(cfm.CapfilmError, match="multiples of 16"):
        cfm._check(L.cf_unet_conv_tc(p(x), 1, 4, 4, 4, 16, p(w), None, 8, 0, 0, p(y), None))


@pytest.mark.parametrize("n,nz,ny,nx,cin,cout", [(1, 4, 6, 8, 16, 16), (2, 5, 3, 7, 32, 48), (1, 6, 6, 6, 48, 16)])
def test_conv_backward(env, n, nz, ny, nx, cin, cout):
    """Input gradient (mirrored, transposed weights through the forward
    kernel), weight and bias gradients (split-K, fixed-order sums), and the
    ReLU mask, against the FP64 backward of the same layer."""
    torch, cfm = env
    L = cfm.load_library()
    rng = np.random.default_rng(100 + cin + cout)
    x = W.bf16_round(rng.standard_normal((n, nz, ny, nx, cin)))
    w = W.bf16_round(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = np.zeros(cout)
    y = W.conv3d_cl(x, w, b, True)
    y16 = W.bf16_round(y)
    g = rng.standard_normal(y.shape).astype(np.float32)
    gm = W.bf16_round(g * (y16 > 0))  # what the kernels see after the ReLU mask
    gx_ref, gw_ref, gb_ref = W.conv3d_cl_backward(x, w, y16, False, gm)
    xd, wd = bf16_dev(torch, x), bf16_dev(torch, w)
    yd = bf16_dev(torch, y16)
    gd = torch.from_numpy(g).cuda()
    gmd = torch.empty(g.size, device="cuda", dtype=torch.bfloat16)
    cfm._check(L.cf_unet_relu_grad(p(gd), None, p(yd), g.size, p(gmd), None))
    torch.cuda.synchronize()
    assert np.array_equal(host(gmd).reshape(gm.shape), gm)
    wt = torch.empty_like(wd)
    cfm._check(L.cf_unet_flip(p(wd), cin, cout, p(wt), None))
    gx = torch.empty(x.size, device="cuda")
    cfm._check(L.cf_unet_conv(p(gmd), n, nz, ny, nx, cout, p(wt), None, cin, 0, 1, p(gx), None))
    chunks = 7
    part = torch.empty(chunks * 27 * cout * cin, device="cuda")
    gw = torch.zeros(27 * cout * cin, device="cuda")
    gb = torch.zeros(cout, device="cuda")
    cfm._check(L.cf_unet_wgrad(p(xd), p(gmd), n, nz, ny, nx, cin, cout, chunks, p(part), p(gw), p(gb), None))
    torch.cuda.synchronize()
    assert rel(host(gx).reshape(x.shape), gx_ref) < 5e-6
    assert rel(host(gw).reshape(gw_ref.shape), gw_ref) < 5e-6
    assert rel(host(gb), gb_ref) < 5e-6
    # bitwise reproducible: a second weight gradient equals the first
    gw2 = torch.zeros_like(gw)
    cfm._check(L.cf_unet_wgrad(p(xd), p(gmd), n, nz, ny, nx, cin, cout, chunks, p(part), p(gw2), None, None))
    torch.cuda.synchronize()
    assert torch.equal(gw, gw2)


def test_pool_upsample_concat_and_layouts(env):
    torch, cfm = env
    L = cfm.load_library()
    rng = np.random.default_rng(5)
    n, nz, ny, nx, c = 2, 4, 6, 8, 16
    x = W.bf16_round(rng.standard_normal((n, nz, ny, nx, c)))
    xd = bf16_dev(torch, x)
    yp = torch.empty(x.size // 8, device="cuda", dtype=torch.bfloat16)
    cfm._check(L.cf_unet_pool(p(xd), n, nz, ny, nx, c, p(yp), None))
    up = torch.empty(x.size, device="cuda", dtype=torch.bfloat16)
    cfm._check(L.cf_unet_upsample(p(yp), n, nz, ny, nx, c, p(up), None))
    g = rng.standard_normal((n, nz // 2, ny // 2, nx // 2, c)).astype(np.float32)
    gf = rng.standard_normal(x.shape).astype(np.float32)
    gd, gfd = torch.from_numpy(g).cuda(), torch.from_numpy(gf).cuda()
    gpool = torch.empty(x.size, device="cuda")
    cfm._check(L.cf_unet_pool_bwd(p(gd), n, nz, ny, nx, c, p(gpool), None))
    gup = torch.empty(x.size // 8, device="cuda")
    cfm._check(L.cf_unet_upsample_bwd(p(gfd), n, nz, ny, nx, c, p(gup), None))
    torch.cuda.synchronize()
    pool_ref = W.avg_pool2(x)
    assert np.abs(host(yp).reshape(pool_ref.shape) - pool_ref).max() <= 2 ** -8 * np.abs(pool_ref).max()
    assert np.array_equal(host(up).reshape(x.shape), W.upsample2(host(yp).reshape(pool_ref.shape)))
    assert np.allclose(host(gpool).reshape(x.shape), W.avg_pool2_backward(g), rtol=1e-7, atol=0)
    assert np.allclose(host(gup).reshape(g.shape), W.upsample2_backward(gf), rtol=1e-6, atol=1e-6)
    # concat / split
    nv = n * nz * ny * nx
    a = W.bf16_round(rng.standard_normal((nv, 16)))
    bb = W.bf16_round(rng.standard_normal((nv, 32)))
    cat = torch.empty(nv * 48, device="cuda", dtype=torch.bfloat16)
    ad, bd = bf16_dev(torch, a), bf16_dev(torch, bb)  # both alive until the kernel has run
    cfm._check(L.cf_unet_concat(nv, p(ad), 16, p(bd), 32, p(cat), None))
    yf = rng.standard_normal((nv, 48)).astype(np.float32)
    sa = torch.empty(nv * 16, device="cuda"); sb = torch.empty(nv * 32, device="cuda")
    yfd = torch.from_numpy(yf).cuda()
    cfm._check(L.cf_unet_split(nv, p(yfd), 16, 32, p(sa), p(sb), None))
    torch.cuda.synchronize()
    assert np.array_equal(host(cat).reshape(nv, 48), np.concatenate([a, bb], axis=1))
    assert np.array_equal(host(sa).reshape(nv, 16), yf[:, :16]) and np.array_equal(host(sb).reshape(nv, 32), yf[:, 16:])
    # pack / unpack (one sample, channel-first float <-> channels-last)
    N = nz * ny * nx
    f = rng.standard_normal((4, N)).astype(np.float32)
    pk = torch.empty(N * 16, device="cuda", dtype=torch.bfloat16)
    fd = torch.from_numpy(f).cuda()
    cfm._check(L.cf_unet_pack(p(fd), 4, N, 16, p(pk), None))
    un = torch.empty(2 * N, device="cuda")
    cfm._check(L.cf_unet_unpack(p(pk), 0, 16, N, 1, 2, p(un), None))
    torch.cuda.synchronize()
    pkh = host(pk).reshape(N, 16)
    assert np.array_equal(pkh[:, :4], W.bf16_round(f.T)) and not pkh[:, 4:].any()
    assert np.array_equal(host(un).reshape(2, N), W.bf16_round(f[1:3]))


def test_bad_shapes_are_rejected(env):
    torch, cfm = env
    L = cfm.load_library()
    a = torch.zeros(1024, device="cuda", dtype=torch.bfloat16)
    assert L.cf_unet_conv(p(a), 1, 2, 2, 2, 12, p(a), None, 8, 0, 0, p(a), None) == 1   # cin not 16k
    assert L.cf_unet_conv(p(a), 1, 2, 2, 2, 16, p(a), None, 6, 0, 0, p(a), None) == 1   # cout not 8k
    assert L.cf_unet_pool(p(a), 1, 3, 2, 2, 16, p(a), None) == 1                         # odd grid


# ------------------------------------------------------------- the whole U-net
def test_unet_forward_backward_match_fp64_composition(env):
    """A small U-net (widths 16, 16, 16) on an 8 x 8 x 12 grid: every
    activation the GPU stores equals the FP64 layer of oracle/warm_net.py
    applied to the GPU's own (bfloat16) input of that layer, rounded to
    bfloat16 (a one-ulp difference allowed where the float32 and FP64 sums
    round differently); the loss kernel matches its definition on the GPU's
    head; and every weight and bias gradient matches the FP64 backward
    composition (skip connections, pooling and upsampling adjoints) fed with
    the GPU's activations and bfloat16-rounded masked gradients."""
    torch, cfm = env
    from paper_2007_15405_gb300 import unet as U
    net = U.UNet(widths=(16, 16, 16), seed=3)
    n, nz, ny, nx = 1, 8, 8, 12
    grid = (n, nz, ny, nx)
    V = nz * ny * nx
    rng = np.random.default_rng(2)
    x = np.zeros((n, nz, ny, nx, 16))
    x[..., :4] = rng.standard_normal((n, nz, ny, nx, 4))
    x = W.bf16_round(x)
    a = net.forward(bf16_dev(torch, x), grid)
    torch.cuda.synchronize()
    A = {k: host(v) for k, v in a.items()}
    Wt = {name: W.bf16_round(net.w[name].cpu().numpy().astype(np.float64)).reshape(27, co, ci)
          for name, ci, co, _ in net.specs}
    Bt = {k: net.b[k].cpu().numpy().astype(np.float64) for k in net.b}
    shp = {"x": (nz, ny, nx), "e0a": (nz, ny, nx), "e0b": (nz, ny, nx), "p1": (4, 4, 6), "e1a": (4, 4, 6),
           "e1b": (4, 4, 6), "p2": (2, 2, 3), "ma": (2, 2, 3), "mb": (2, 2, 3), "u1": (4, 4, 6),
           "c1": (4, 4, 6), "d1a": (4, 4, 6), "d1b": (4, 4, 6), "u0": (nz, ny, nx), "c0": (nz, ny, nx),
           "d0a": (nz, ny, nx), "d0b": (nz, ny, nx), "head": (nz, ny, nx)}
    A = {k: v.reshape((n,) + shp[k] + (-1,)) for k, v in A.items()}
    inputs = {"e0a": "x", "e0b": "e0a", "e1a": "p1", "e1b": "e1a", "ma": "p2", "mb": "ma", "d1a": "c1",
              "d1b": "d1a", "d0a": "c0", "d0b": "d0a", "head": "d0b"}
    for name, _, _, relu in net.specs:
        ref = W.conv3d_cl(A[inputs[name]], Wt[name], Bt[name], relu)
        if name != "head":
            ref = W.bf16_round(ref)
        err = np.abs(A[name] - ref).max()
        assert err <= 2 ** -7 * np.abs(ref).max() + 1e-6, (name, err)
    assert np.abs(A["p1"] - W.bf16_round(W.avg_pool2(A["e0b"]))).max() <= 2 ** -7 * np.abs(A["p1"]).max()
    assert np.array_equal(A["u1"], W.upsample2(A["mb"]))
    assert np.array_equal(A["c1"], np.concatenate([A["e1b"], A["u1"]], axis=-1))
    assert np.array_equal(A["c0"], np.concatenate([A["e0b"], A["u0"]], axis=-1))
    # loss: density part and displacement part at a few nodes
    t = rng.standard_normal((n, 2, V)).astype(np.float32) * 0.1
    mask = (rng.random((n, V)) > 0.3).astype(np.float32)
    Xn = (rng.random((n, 5, 3)) * np.array([nx - 1, ny - 1, nz - 1])).astype(np.float32)
    dn = rng.standard_normal((n, 5, 3)).astype(np.float32) * 0.05
    msum = float(mask.sum())
    td, md = torch.from_numpy(t).cuda(), torch.from_numpy(mask).cuda()
    Xd, dd = torch.from_numpy(Xn).cuda(), torch.from_numpy(dn).cuda()
    loss, g = net.loss_and_grad(a, grid, td, md, msum, Xd, dd, 5, wd=1.0, wx=0.5)
    torch.cuda.synchronize()
    H = A["head"][0].reshape(V, 16)
    Ld = np.sum(mask[0][:, None] * (H[:, :2] - t[0].T) ** 2) / msum
    Lx = 0.0
    Gref = np.zeros((V, 16))
    Gref[:, :2] = 2 * mask[0][:, None] * (H[:, :2] - t[0].T) / msum
    for i in range(5):
        px, py, pz = Xn[0, i].astype(np.float64)
        x0, y0, z0 = int(px), int(py), int(pz)
        fx, fy, fz = px - x0, py - y0, pz - z0
        D = np.zeros(3)
        corners = []
        for k in range(8):
            ddx, ddy, ddz = k & 1, (k >> 1) & 1, k >> 2
            wgt = (fx if ddx else 1 - fx) * (fy if ddy else 1 - fy) * (fz if ddz else 1 - fz)
            v = ((z0 + ddz) * ny + (y0 + ddy)) * nx + (x0 + ddx)
            corners.append((v, wgt))
            D += wgt * H[v, 2:5]
        r = D - dn[0, i]
        Lx += 0.5 / 5 * np.sum(r * r)
        for v, wgt in corners:
            Gref[v, 2:5] += 2 * 0.5 / 5 * wgt * r
    assert float(loss.item()) == pytest.approx(Ld + Lx, rel=1e-5)
    assert np.abs(host(g).reshape(V, 16) - Gref).max() <= 1e-5 * np.abs(Gref).max()
    # backward against the FP64 composition on the GPU's activations
    grads = net.backward(a, g, grid)
    torch.cuda.synchronize()
    G = host(g).reshape((n,) + shp["head"] + (16,))
    ref_gw = {}

    def back(name, gy, gy2=None):
        relu = net._spec(name)[3]
        gsum = gy + (gy2 if gy2 is not None else 0.0)
        gm = W.bf16_round(gsum * (A[name] > 0) if relu else gsum)
        gx, gw, gb = W.conv3d_cl_backward(A[inputs[name]], Wt[name], A[name], False, gm)
        ref_gw[name] = (gw, gb)
        return gx

    gd0b = back("head", G)
    gd0a = back("d0b", gd0b)
    gc0 = back("d0a", gd0a)
    ge0b_skip, gu0 = gc0[..., :16], gc0[..., 16:]
    gd1a = back("d1b", W.upsample2_backward(gu0))
    gc1 = back("d1a", gd1a)
    ge1b_skip, gu1 = gc1[..., :16], gc1[..., 16:]
    gma = back("mb", W.upsample2_backward(gu1))
    gp2 = back("ma", gma)
    ge1a = back("e1b", ge1b_skip, W.avg_pool2_backward(gp2))
    gp1 = back("e1a", ge1a)
    ge0a = back("e0b", ge0b_skip, W.avg_pool2_backward(gp1))
    back("e0a", ge0a)
    # the reference carries the input gradients in FP64, the GPU in float32:
    # where a masked gradient sits at a bfloat16 rounding boundary the two
    # round it one ulp (2^-8) apart, so the bound is on the bfloat16 scale
    for name in net.w:
        gw, gb = grads[name]
        rw, rb = ref_gw[name]
        rw = rw.reshape(-1)
        assert np.abs(host(gw) - rw).max() <= 1e-2 * np.abs(rw).max() + 1e-9, name
        assert np.abs(host(gb) - rb).max() <= 1e-2 * np.abs(rb).max() + 1e-9, name


def test_unet_training_is_reproducible_and_learns(env):
    """Two trainings from the same seed on the same data give bitwise equal
    weights (fixed-order sums everywhere), and the loss falls."""
    torch, cfm = env
    from paper_2007_15405_gb300 import unet as U
    n, nz, ny, nx = 2, 8, 8, 8
    V = nz * ny * nx
    rng = np.random.default_rng(4)
    x = np.zeros((n, nz, ny, nx, 16))
    x[..., :4] = rng.standard_normal((n, nz, ny, nx, 4))
    xd = bf16_dev(torch, W.bf16_round(x))
    t = torch.from_numpy((0.3 * np.tanh(x[..., :2])).transpose(0, 4, 1, 2, 3).reshape(n, 2, V)
                         .astype(np.float32)).cuda()
    m = torch.ones(n * V, device="cuda")
    out = []
    for rep in range(2):
        net = U.UNet(widths=(16, 16, 16), seed=1)
        losses = [net.train_step(xd, (n, nz, ny, nx), t, m, float(n * V), lr=3e-3) for _ in range(40)]
        out.append((losses, {k: v.clone() for k, v in net.w.items()}))
    assert out[0][0] == out[1][0]
    assert all(torch.equal(out[0][1][k], out[1][1][k]) for k in out[0][1])
    assert out[0][0][-1] < 0.5 * out[0][0][0]


# ---------------------------------------------------- the library's warm start
def test_library_warm_start_equals_python_path_and_falls_back(env, tmp_path):
    """cf_model_load + cf_warmstart (inference, predicted state and judging
    inside the library) give bitwise the state of the Python orchestration of
    the same kernels (features, U-net, cf_warm_apply, the same judging
    steps); a policy that cannot be met restores the flat film."""
    torch, cfm = env
    from paper_2007_15405_gb300 import inputs as I, unet as U, warm
    wl = I.warm_pair_dataset(1, seed=3, nx=48, ny=32, nz=32, radius=5.0, level=2)[0]
    net = U.UNet(widths=(16, 32, 32), seed=5)
    path = str(tmp_path / "unet.bin")
    net.save(path)
    model = cfm.Model(path)
    a = cfm.Simulation.from_workload(wl, set_film=False)
    used, steps = a.warmstart(model, wl.h_top, wl.capsules[0].kS, window=10, u_limit=1.0, grow=1e9)
    assert used and steps == 21
    b = cfm.Simulation.from_workload(wl, set_film=False)
    x, _ = warm.features_dev(b, wl)
    d = net.predict_dev(x, (wl.nz, wl.ny, wl.nx))
    b.warm_apply(wl.h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, d)
    b.step(1); b.field_check(); b.step(10); b.field_check(); b.step(10); b.field_check()
    assert np.array_equal(a.populations(), b.populations())
    # a velocity limit nothing meets: back to the flat film
    c = cfm.Simulation.from_workload(wl, set_film=False)
    used, _ = c.warmstart(model, wl.h_top, wl.capsules[0].kS, jitter=wl.jitter(), window=5, u_limit=1e-30)
    assert not used
    f = cfm.Simulation.from_workload(wl)
    assert np.array_equal(c.populations(), f.populations())
    model.close()
