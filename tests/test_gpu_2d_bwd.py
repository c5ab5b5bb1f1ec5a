"""GPU parity of the 2D greedy forward and of the 1D adjoint (plus its autograd wrapper)."""
import numpy as np
import pytest
import torch

import synth
from hs_check import compare_argmax, compare_form, path_view

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


# ---------------------------------------------------------------------------------------------
# 2D greedy
# ---------------------------------------------------------------------------------------------
def run_2d(hs, o, pl, z0, H, flags=0, mean1=2.0, order=None, dtype=0, tuning=None, default_kernel=None):
    """dtype 1 / 2: the plane is rounded to FP16 / BF16 on the host (round to nearest even) and
    the oracle runs on the rounded values, which FP32 holds exactly.  ``order`` picks kernel 0 or
    1; ``tuning`` sets any launch shape (the column sweep: kernel 2); ``default_kernel``: the
    kernel the plan's default launch shape must name."""
    n_rows, n_freq = pl.shape
    if dtype:
        t = torch.from_numpy(pl).to({1: torch.float16, 2: torch.bfloat16}[dtype])
        pl_dev, pl = t.to(DEV), t.float().numpy()
    else:
        pl_dev = torch.from_numpy(pl).to(DEV)
    plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=n_rows, z0_row=z0, flags=flags, dtype=dtype)
    if order is not None:
        plan.tuning = dict(kernel=order, threads=256)     # 0: f-tiles fastest, 1: z rows fastest
        assert plan.tuning.kernel == order
    if tuning is not None:
        plan.tuning = tuning
        assert plan.tuning.kernel == tuning["kernel"]
    if default_kernel is not None:
        assert plan.tuning.kernel == default_kernel
    assert plan.domain == o.domain_2d(n_freq, n_rows, z0, H)
    mu, sg = hs.norm_exponential(2, 2, H, True, mean1)
    ng = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    out = plan.forward(pl_dev, None, ng)[hs.GREEDY]
    torch.cuda.synchronize()
    hs.check_device_error(plan)
    r_snr, r_bh, r_path, r_all = o.greedy_2d(pl, z0, H, mu, sg, want_all=True)
    g_snr = out.snr.cpu().numpy()
    near = compare_form(g_snr, out.best_h.cpu().numpy(), r_snr, r_bh, r_all, mu, sg,
                        path_view(out.path, H), r_path, what="2d")
    compare_argmax(out.argmax.cpu().numpy()[0], r_snr, g_snr, mu, sg, r_bh, hs.decode_argmax, what="2d argmax")
    plan.close()
    return near


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("H", [1, 2, 3, 4, 8])
def test_2d_small(hs, oracle_lib, H, order):
    z0 = 30
    pl = synth.plane(5003, 2 * z0 + 1, z0, 40 + H, synth.random_tracks(3, 5003, 8, f_lo=50, zmax=3))
    run_2d(hs, oracle_lib, pl, z0, H, order=order)


def test_2d_asymmetric_rows_checked(hs, oracle_lib):
    pl = synth.plane(3001, 37, 14, 3)
    run_2d(hs, oracle_lib, pl, 14, 4, flags=hs.FLAG_CHECKED)


def test_2d_integer_ties(hs, oracle_lib):
    pl = np.floor(synth.plane(2048, 41, 20, 6) * 0.7).astype(np.float32)
    run_2d(hs, oracle_lib, pl, 20, 5)


@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("H", [3, 8])
def test_2d_reduced_precision(hs, oracle_lib, H, dtype):
    """FP16 / BF16 plane storage: comparisons on the stored values, FP32 sums."""
    z0 = 30
    pl = synth.plane(5003, 2 * z0 + 1, z0, 70 + H, synth.random_tracks(3, 5003, 18, f_lo=50, zmax=3))
    for order in (0, 1):
        run_2d(hs, oracle_lib, pl, z0, H, order=order, dtype=dtype)


def test_2d_integer_ties_bf16(hs, oracle_lib):
    """Small integers are exact in BF16: dense ties exercise the strict raster-order rule."""
    pl = np.floor(synth.plane(2048, 41, 20, 9) * 0.7).astype(np.float32)
    run_2d(hs, oracle_lib, pl, 20, 5, dtype=2, flags=hs.FLAG_CHECKED)


def test_2d_full_size(hs, oracle_lib):
    """f-fdot plane 201 x 2^21, H = 8, chi-square(2) noise + 8 drifting tracks: kernels 0 and 1,
    the column sweep in its default launch (the FP32 default for a plane this size) and at 512
    threads, and the FP16 plane (kernel 1 by default)."""
    tracks = synth.random_tracks(8, synth.PLANE_N_FREQ, synth.SEED_BASE + 4 + 1000)
    pl = synth.plane(synth.PLANE_N_FREQ, synth.PLANE_N_ROWS, synth.PLANE_Z0_ROW, synth.SEED_BASE + 4, tracks)
    for order in (0, 1):
        near = run_2d(hs, oracle_lib, pl, synth.PLANE_Z0_ROW, 8, order=order)
        assert near <= 20
    near = run_2d(hs, oracle_lib, pl, synth.PLANE_Z0_ROW, 8, default_kernel=2)
    assert near <= 20
    near = run_2d(hs, oracle_lib, pl, synth.PLANE_Z0_ROW, 8, tuning=dict(kernel=2, threads=512))
    assert near <= 20
    near = run_2d(hs, oracle_lib, pl, synth.PLANE_Z0_ROW, 8, dtype=1, default_kernel=1)
    assert near <= 20


# ---------------------------------------------------------------------------------------------
# 1D adjoint
# ---------------------------------------------------------------------------------------------
def bwd_case(hs, o, xs, H, form, w=None, dtype=0, mitigation=True, sparse=0):
    """Adjoint against the FP64 oracle; ``sparse`` > 0 keeps that many nonzero upstream
    gradients per spectrum (as a top-k loss does) and zeroes the rest."""
    lengths = [len(x) for x in xs]
    flags = (hs.FLAG_WHITENING if w is not None else 0) | (0 if mitigation else hs.FLAG_NO_MITIGATION)
    plan = hs.Plan(H, form, lengths=lengths, dtype=dtype, flags=flags)
    tdt = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[dtype]
    buf = torch.zeros(plan.extent, dtype=tdt)
    refs = []
    for s, x in enumerate(xs):
        t = torch.from_numpy(x).to(tdt)
        buf[int(plan.input_offsets[s]):int(plan.input_offsets[s]) + len(x)] = t
        refs.append(t.float().numpy())
    xd = buf.to(DEV)
    wd = None if w is None else torch.from_numpy(w).to(DEV)
    mu, sg = hs.norm_exponential(form, 1, H, mitigation)
    nrm = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    out = plan.forward(xd, nrm if form == 1 else None, nrm if form == 2 else None, w=wd)[form]
    gh = synth.upstream_grad(plan.total_fundamentals, 17)
    if sparse:
        keep = np.zeros(gh.size, bool)
        rng = np.random.default_rng(99)
        for s in range(len(xs)):
            a, b = int(plan.fund_offsets[s]), int(plan.fund_offsets[s + 1])
            keep[rng.choice(np.arange(a, b), size=min(sparse, b - a), replace=False)] = True
        gh = np.where(keep, gh, np.float32(0.0)).astype(np.float32)
    g = torch.from_numpy(gh).to(DEV)
    gin = torch.zeros(plan.extent, dtype=torch.float32, device=DEV)
    gw = torch.zeros(len(xs[0]), dtype=torch.float32, device=DEV) if w is not None else None
    hs.backward(plan, form, g, out, xd, wd, gin, gw)
    gin2 = torch.zeros_like(gin)
    gw2 = torch.zeros_like(gw) if gw is not None else None
    hs.backward(plan, form, g, out, xd, wd, gin2, gw2)
    torch.cuda.synchronize()
    assert torch.equal(gin, gin2), "adjoint is not bit-reproducible"
    if gw is not None:
        assert torch.equal(gw, gw2)
    else:
        # without the workspace every block is visited: the same bits as with block marking
        gin3 = torch.zeros_like(gin)
        hs.backward(plan, form, g, out, xd, wd, gin3, None, mark_blocks=False)
        torch.cuda.synchronize()
        assert torch.equal(gin, gin3), "block marking changed the adjoint"
    gin = gin.cpu().numpy()
    gn = g.cpu().numpy().astype(np.float64)
    gw_ref = np.zeros(len(xs[0])) if w is not None else None
    for s, x in enumerate(xs):
        a, b = int(plan.fund_offsets[s]), int(plan.fund_offsets[s + 1])
        if form == 1:
            r_snr, r_bh = o.simple_1d(refs[s], H, mu, sg, w=w)
            r_path = None
        else:
            r_snr, r_bh, r_path = o.greedy_1d(refs[s], H, mu, sg, mitigation=mitigation, w=w)
        # the adjoint is defined by the forward's choices: require identical ones here
        assert np.array_equal(out.best_h.cpu().numpy()[a:b], r_bh)
        gx_ref = o.backward_1d(form, len(x), H, r_bh, sg, gn[a:b], r_path)
        off = int(plan.input_offsets[s])
        got = gin[off:off + len(x)].astype(np.float64)
        want = gx_ref * (w.astype(np.float64) if w is not None else 1.0)
        scale = np.abs(gn[a:b]).max() / sg.min() * H
        np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * scale)
        if w is not None:
            gw_ref += refs[s].astype(np.float64) * gx_ref
    if w is not None:
        scale = np.abs(gw_ref).max()
        np.testing.assert_allclose(gw.cpu().numpy(), gw_ref, rtol=1e-5, atol=1e-6 * scale)
    plan.close()


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("H", [1, 5, 16, 32])
def test_backward_single(hs, oracle_lib, form, H):
    x = synth.spectrum(50001, 3 + H, [synth.Pulsar(401.2, 0.05)])
    bwd_case(hs, oracle_lib, [x], H, form)


@pytest.mark.parametrize("form", [1, 2])
def test_backward_sparse_gradient(hs, oracle_lib, form):
    """A few nonzero upstream gradients per spectrum over uneven lengths: most bin blocks receive
    nothing and are skipped."""
    xs = [synth.spectrum(n, 40 + n % 97, [synth.Pulsar(77.7, 0.05)]) for n in (70001, 4099, 33, 1 << 17)]
    bwd_case(hs, oracle_lib, xs, 32, form, sparse=16)
    bwd_case(hs, oracle_lib, xs, 7, form, sparse=3)


@pytest.mark.parametrize("dtype", [0, 2])
def test_backward_sparse_whitening(hs, oracle_lib, dtype):
    N = 1 << 15
    w = synth.whitening(N, 4)
    xs = [synth.spectrum(N, 80 + i, [synth.Pulsar(150.3 + i, 0.05)]) for i in range(5)]
    bwd_case(hs, oracle_lib, xs, 32, 2, w=w, dtype=dtype, sparse=16)


def test_backward_unmitigated_batch(hs, oracle_lib):
    xs = [synth.spectrum(n, n) for n in (4099, 10000, 33, 70000)]
    bwd_case(hs, oracle_lib, xs, 8, 2, mitigation=False)


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_backward_whitening(hs, oracle_lib, dtype):
    N = 1 << 15
    w = synth.whitening(N, 2)
    xs = [synth.spectrum(N, 60 + i, [synth.Pulsar(150.3 + i, 0.05)]) for i in range(4)]
    bwd_case(hs, oracle_lib, xs, 32, 2, w=w, dtype=dtype)
    bwd_case(hs, oracle_lib, xs, 16, 1, w=w, dtype=dtype)


def test_backward_whitening_many_groups(hs, oracle_lib):
    """More spectra than dL/dw partial groups: each group sums several spectra, then the groups
    are added in order."""
    N = 4096
    w = synth.whitening(N, 9)
    xs = [synth.spectrum(N, 700 + i, [synth.Pulsar(40.3 + i, 0.05)]) for i in range(20)]
    bwd_case(hs, oracle_lib, xs, 16, 2, w=w)


def test_autograd_topk_loss_matches_fd(hs, oracle_lib):
    """loss = -sum of the top-16 greedy SNRs per spectrum, learnable whitening w (init 1.0):
    the adjoint's dL/dw matches central finite differences (eps = 1e-3) of the FP64 oracle on a
    4096-bin slice and the oracle's analytic gradient everywhere."""
    B, N, H, K = 4, 1 << 16, 32, 16
    pulsars = [synth.Pulsar(200.0 + 37.3 * i, 0.05) for i in range(B)]
    ps = [synth.spectrum(N, 300 + i, [pulsars[i]]) for i in range(B)]
    p = torch.from_numpy(np.concatenate(ps)).to(DEV)
    w = torch.ones(N, device=DEV, requires_grad=True)
    plan = hs.Plan(H, hs.GREEDY, lengths=[N] * B, flags=hs.FLAG_WHITENING)
    mu, sg = hs.norm_exponential(2, 1, H)
    nrm = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    snr, bh, path = hs.HarmonicSum.apply(p, w, plan, hs.GREEDY, *nrm)
    nf = plan.total_fundamentals // B
    loss = -snr.view(B, nf).topk(K, dim=1).values.sum()
    loss.backward()
    gw = w.grad.cpu().numpy().astype(np.float64)

    o = oracle_lib
    w0 = np.ones(N, np.float32)

    def oracle_loss(wv, round_w=True):
        tot = 0.0
        choice = []
        for x in ps:
            s, b, pa = o.greedy_1d(x, H, mu, sg, w=wv, round_w=round_w)
            top = np.argsort(-s, kind="stable")[:K]
            tot -= s[top].sum()
            choice.append((b, pa, top))
        return tot, choice

    L0, choice0 = oracle_loss(w0)
    gw_ref = np.zeros(N)
    for (b, pa, top), x in zip(choice0, ps):
        g = np.zeros(nf)
        g[top] = -1.0
        gw_ref += x.astype(np.float64) * o.backward_1d(2, N, H, b, sg, g, pa)
    np.testing.assert_allclose(gw, gw_ref, rtol=1e-5, atol=1e-6)
    # central differences on a 4096-bin slice holding the pulsars' harmonics
    j0 = 0                                  # bins 0..4095 hold harmonics of every pulsar
    eps = 1e-3
    js = list(range(j0, j0 + 4096))
    sel = [j for j in js if gw_ref[j] != 0.0] + js[::256]
    checked = 0
    for j in sel:
        wp, wm = w0.copy(), w0.copy()
        wp[j] += eps
        wm[j] -= eps
        Lp, cp = oracle_loss(wp, round_w=False)
        Lm, cm = oracle_loss(wm, round_w=False)
        if any(not (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]))
               for a, b in zip(cp, cm)):
            continue          # a discrete choice flipped inside +-eps: FD is not a derivative here
        dw = float(np.float32(wp[j])) - float(np.float32(wm[j]))
        fd = (Lp - Lm) / dw
        assert abs(fd - gw[j]) <= 1e-4 * max(1.0, abs(fd)), (j, fd, gw[j])
        checked += 1
    assert checked >= 16


def _f32_nearest(num: int, e2: int) -> np.float32:
    """The float32 nearest to num * 2^e2 (ties to even), from exact rational arithmetic."""
    from fractions import Fraction
    exact = Fraction(num) * (Fraction(2) ** e2)
    x0 = np.float32(float(exact))
    best = None
    for c in (np.nextafter(x0, np.float32(-np.inf)), x0, np.nextafter(x0, np.float32(np.inf))):
        err = abs(Fraction(float(c)) - exact)
        key = (err, int(np.array(c, np.float32).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


@pytest.mark.parametrize("form", [1, 2])
def test_backward_fixed_point_bit_exact(hs, oracle_lib, form):
    """hs_backward's rounding rule, bit for bit: contributions c = fl32(g * fl32(1/sigma)) are
    scaled to integers round(c * 2^(55 - e)), e the exponent of the largest |c| of the 1024-bin
    block, summed exactly, and each bin's sum is rounded once to FP32."""
    N, H, L = 30011, 32, 1024
    x = synth.spectrum(N, 5 + form, [synth.Pulsar(123.4, 0.05)])
    plan = hs.Plan(H, form, lengths=[N])
    mu, sg = hs.norm_exponential(form, 1, H)
    nrm = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    xd = torch.from_numpy(x).to(DEV)
    out = plan.forward(xd, nrm if form == 1 else None, nrm if form == 2 else None)[form]
    g = synth.upstream_grad(plan.total_fundamentals, 23)
    gin = torch.zeros(plan.extent, dtype=torch.float32, device=DEV)
    hs.backward(plan, form, torch.from_numpy(g).to(DEV), out, xd, None, gin, None)
    torch.cuda.synchronize()
    got = gin.cpu().numpy()[:N]
    if form == 1:
        _, bh = oracle_lib.simple_1d(x, H, mu, sg)
        path = np.zeros(bh.size, np.uint64)
    else:
        _, bh, path = oracle_lib.greedy_1d(x, H, mu, sg)
        path = path.astype(np.uint64)
    assert np.array_equal(out.best_h.cpu().numpy(), bh)
    rs = (np.float32(1.0) / sg.astype(np.float32)).astype(np.float32)
    n = np.arange(bh.size, dtype=np.int64)
    bins, vals = [], []
    for k in range(1, H + 1):
        sel = bh >= k
        drift = np.zeros(bh.size, np.int64)
        if form == 2:
            mask = np.uint64((1 << k) - 1)
            drift = np.array([bin(int(p & mask)).count("1") for p in path], np.int64)
        bins.append((k * n + drift)[sel])
        vals.append((g[sel].astype(np.float32) * rs[bh[sel] - 1]).astype(np.float32))
    bins, vals = np.concatenate(bins), np.concatenate(vals)
    blk = bins // L
    vmax = np.zeros(N // L + 1)
    np.maximum.at(vmax, blk, np.abs(vals.astype(np.float64)))
    ex = np.frexp(vmax)[1] - 1                     # exponent e with 2^e <= vmax < 2^(e+1)
    fixed = np.rint(vals.astype(np.float64) * np.ldexp(1.0, 55 - ex[blk])).astype(np.int64)
    acc = np.zeros(N, np.int64)
    np.add.at(acc, bins, fixed)
    want = np.zeros(N, np.float32)
    for j in np.nonzero(acc)[0]:
        want[j] = _f32_nearest(int(acc[j]), int(ex[j // L]) - 55)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), \
        f"{np.count_nonzero(got.view(np.uint32) != want.view(np.uint32))} bins differ"
    plan.close()
