"""Parity of the CUDA soft layer (dp_pix_soft_forward / dp_pix_soft_backward, through the C ABI and the
autograd wrapper) with the fp64 oracle, element by element on seeded inputs.

Tolerances follow from the arithmetic.  A noisy mean pre = S/b^2 + eta is compared with the rule used for
the release: |pre_gpu - pre_ora| <= 2e-5 max(|pre|, |mu|, |eta|).  y = w p0 + (1 - w) p1 inherits
w err0 + (1 - w) err1 plus one f32 rounding.  Gradients are sums of f32 products over at most b^2 pixels:
the bound is 2e-5 times the same sums taken over absolute values, plus 1e-7.  Where a noisy mean lies
within that bound of 0 or R the clip decision may legitimately differ; such cells are left out of the
gradient comparison (and counted)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2511_04261_b300 as P

pytestmark = pytest.mark.gpu
REL = 2e-5


def _inputs(B, C, H, W, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    x = np.empty((B, C, H, W), np.float32)
    w = np.empty((B, 1, H, W), np.float32)
    for n in range(B):
        for c in range(C):
            base = rng.uniform(0.1, 0.5) + rng.uniform(-0.2, 0.3) * xx / max(1, W - 1)
            x[n, c] = np.clip(base + rng.normal(0, 0.15, size=(H, W)), 0, 1)
        cy, cx = rng.uniform(0.3, 0.7) * H, rng.uniform(0.3, 0.7) * W
        d = np.hypot((yy - cy) / (0.3 * H), (xx - cx) / (0.3 * W))
        w[n, 0] = 1.0 / (1.0 + np.exp((d - 1.0) * 8.0))
    g = rng.normal(size=(B, C, H, W)).astype(np.float32)
    return x, w, g


def _oracle_pre(x, spec, n_frame):
    """(mu, eta) per grid for one image x [C, H, W] (fp64): block means of the mirror-padded planes and the
    oracle's Laplace draws for the layer's counters."""
    C, H, W = x.shape
    out = []
    mode = "reflect" if spec.pad_mode == 0 else "symmetric"
    for j, b in enumerate(spec.grids):
        gr, gc = -(-H // b), -(-W // b)
        xp = np.pad(x.astype(np.float64), ((0, 0), (0, gr * b - H), (0, gc * b - W)), mode=mode)
        mu = xp.reshape(C, gr, b, gc, b).mean(axis=(2, 4))
        eta = np.zeros_like(mu)
        if not spec.noise_free:
            sigma = spec.R * spec.m / (b * b * spec.eps[j])
            frame = spec.frame0 + n_frame
            key = [spec.seed & 0xFFFFFFFF, spec.seed >> 32]
            for cy in range(gr):
                for cx in range(gc):
                    wd = O.philox4x32_10([cy * gc + cx, j | (spec.stream_id << 8), frame & 0xFFFFFFFF, frame >> 32], key)
                    for c in range(C):
                        eta[c, cy, cx] = O.laplace_from_word(int(wd[c]), sigma)
        out.append((mu, eta))
    return out


def _split_pre(pre, B, C, H, W, grids):
    pre = pre.cpu().numpy().astype(np.float64)
    res, off = [], 0
    dims = [(-(-H // b), -(-W // b)) for b in grids]
    per = sum(C * a * b for a, b in dims)
    for n in range(B):
        img, o = [], n * per
        for (gr, gc) in dims:
            img.append(pre[o:o + C * gr * gc].reshape(C, gr, gc))
            o += C * gr * gc
        res.append(img)
    return res


def _up(a, b, H, W):
    return np.repeat(np.repeat(a, b, axis=-2), b, axis=-1)[..., :H, :W]


def _check(B, C, H, W, grids, eps=(0.5, 1.0), pad_mode=0, noise_free=False, seed=1, frame0=0, images=None):
    spec = P.SoftSpec(grids=grids, eps=eps, R=1.0, m=16.0, pad_mode=pad_mode, noise_free=noise_free, seed=seed,
                      frame0=frame0, stream_id=3)
    x, w, g = _inputs(B, C, H, W, seed + H + W)
    xt, wt, gt = (torch.from_numpy(a).cuda() for a in (x, w, g))
    y, pre = P.soft_forward(xt, wt, spec)
    dx, dw = P.soft_backward(wt, gt, pre, spec)
    torch.cuda.synchronize()
    y, dx, dw = y.cpu().numpy(), dx.cpu().numpy(), dw.cpu().numpy()
    pres = _split_pre(pre, B, C, H, W, grids)
    kw = dict(grids=grids, eps=eps, R=1.0, m=16.0, pad_mode=pad_mode, noise_free=noise_free, stream_id=3, seed=seed)
    skipped = 0
    for n in (images if images is not None else range(B)):
        parts = _oracle_pre(x[n], spec, n)
        yo, po = O.soft_forward(x[n:n + 1], w[n:n + 1], frame0=frame0 + n, **kw)
        dxo, dwo = O.soft_backward(x[n:n + 1], w[n:n + 1], g[n:n + 1], frame0=frame0 + n, **kw)
        bounds, ambiguous = [], np.zeros((H, W), bool)
        for j, b in enumerate(grids):
            mu, eta = parts[j]
            pre_o = mu + eta
            # the test's own block means and draws agree with the oracle's broadcast clipped means
            assert np.allclose(_up(np.clip(pre_o, 0, 1), b, H, W), po[0, j], atol=1e-12)
            bound = REL * np.maximum(np.maximum(np.abs(pre_o), np.abs(mu)), np.abs(eta)) + 1e-7
            assert np.all(np.abs(pres[n][j] - pre_o) <= bound), (n, j, float(np.abs(pres[n][j] - pre_o).max()))
            bounds.append(bound)
            amb = (np.abs(pre_o) <= bound).any(axis=0) | (np.abs(pre_o - 1.0) <= bound).any(axis=0)
            ambiguous |= _up(amb, b, H, W)
        # forward
        e0, e1 = _up(bounds[0], grids[0], H, W), _up(bounds[1], grids[1], H, W)
        ybound = w[n, 0] * e0 + (1 - w[n, 0]) * e1 + 2e-7
        assert np.all(np.abs(y[n] - yo[0]) <= ybound), float(np.abs(y[n] - yo[0]).max())
        # dw = sum_ch g (p0 - p1)
        dwb = (np.abs(g[n]) * (e0 + e1)).sum(axis=0) + REL * (np.abs(g[n]) * 2).sum(axis=0) + 1e-7
        assert np.all(np.abs(dw[n, 0] - dwo[0, 0]) <= dwb), float(np.abs(dw[n, 0] - dwo[0, 0]).max())
        # dx, away from cells whose clip decision is within rounding
        gab = np.abs(g[n].astype(np.float64))
        mag = np.zeros_like(gab)
        for j, b in enumerate(grids):
            wj = w[n, 0] if j == 0 else 1 - w[n, 0]
            gr, gc = -(-H // b), -(-W // b)
            s = np.zeros((C, gr * b, gc * b))
            s[:, :H, :W] = gab * wj
            cs = s.reshape(C, gr, b, gc, b).sum(axis=(2, 4)) / (b * b)
            mag += 4 * _up(cs, b, H, W)  # a pixel is read by at most 4 padded samples per grid
        ok = ~ambiguous
        skipped += int((~ok).sum())
        diff = np.abs(dx[n] - dxo[0])[:, ok]
        assert np.all(diff <= (REL * mag + 1e-7)[:, ok]), float(diff.max())
    return skipped


@pytest.mark.parametrize("B,C,H,W,grids", [
    (2, 3, 32, 128, (8, 16)),      # fast path
    (2, 3, 64, 256, (16, 8)),      # fast path, the w-weighted grid is the larger one
    (1, 1, 16, 128, (4, 16)),      # fast path, C = 1
    (1, 4, 32, 128, (8, 32)),      # fast path, C = 4
    (1, 3, 16, 128, (16, 16)),     # fast path, equal grids (two independent releases)
])
def test_soft_fast_path_matches_oracle(B, C, H, W, grids):
    _check(B, C, H, W, grids)


@pytest.mark.parametrize("B,C,H,W,grids,pad", [
    (2, 3, 37, 45, (8, 16), 0),    # mirror padding (reflect)
    (1, 3, 37, 45, (8, 16), 1),    # symmetric padding
    (1, 3, 40, 60, (6, 20), 0),    # grids that are not powers of two
    (1, 2, 33, 128, (8, 16), 0),   # rows need padding, columns do not
    (1, 3, 16, 100, (4, 8), 0),    # W not a multiple of 128
])
def test_soft_generic_path_matches_oracle(B, C, H, W, grids, pad):
    _check(B, C, H, W, grids, pad_mode=pad)


def test_soft_noise_free_and_frame_offset():
    _check(1, 3, 32, 128, (8, 16), noise_free=True)
    _check(2, 3, 32, 128, (8, 16), frame0=2**33 + 5)


def test_soft_autograd_matches_direct_calls_and_finite_differences():
    spec = P.SoftSpec(grids=(8, 16), eps=(0.5, 1.0), R=1.0, m=16.0, seed=9)
    x, w, g = _inputs(1, 3, 32, 128, 4)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    gt = torch.from_numpy(g).cuda()
    y = P.soft_pixelize(xt, wt, spec)
    (y * gt).sum().backward()
    y2, pre = P.soft_forward(xt.detach(), wt.detach(), spec)
    dx2, dw2 = P.soft_backward(wt.detach(), gt, pre, spec)
    assert torch.equal(y, y2) and torch.equal(xt.grad, dx2) and torch.equal(wt.grad, dw2)
    # central differences of L = sum g y on the GPU, per coordinate, from the change of y alone
    # (f32: y changes by ~1e-5 against an ulp of 6e-8, so a 2 % tolerance)
    h = 1e-3
    rng = np.random.default_rng(0)
    for _ in range(6):
        c, i, j = int(rng.integers(0, 3)), int(rng.integers(0, 32)), int(rng.integers(0, 128))
        xp, xm = xt.detach().clone(), xt.detach().clone()
        xp[0, c, i, j] += h
        xm[0, c, i, j] -= h
        yp, pp = P.soft_forward(xp, wt.detach(), spec)
        ym, pm = P.soft_forward(xm, wt.detach(), spec)
        # skip coordinates whose cells change clip state within +-h
        if not torch.equal((pp > 0) & (pp < 1), (pm > 0) & (pm < 1)):
            continue
        fd = float(((yp - ym).double() * gt.double()).sum()) / (2 * h)
        an = float(xt.grad[0, c, i, j])
        assert abs(fd - an) <= 2e-2 * abs(an) + 2e-3, (c, i, j, fd, an)
        wp_, wm_ = wt.detach().clone(), wt.detach().clone()
        wp_[0, 0, i, j] += h
        wm_[0, 0, i, j] -= h
        fdw = float(((P.soft_forward(xt.detach(), wp_, spec)[0] - P.soft_forward(xt.detach(), wm_, spec)[0]).double()
                     * gt.double()).sum()) / (2 * h)
        anw = float(wt.grad[0, 0, i, j])
        assert abs(fdw - anw) <= 2e-2 * abs(anw) + 2e-3, (i, j, fdw, anw)


def test_soft_full_size_batch_sampled():
    """The benchmark shape (32 x 3 x 1024 x 1024, grids 8 and 16) in the launch configuration the benchmark
    uses; images 0 and 31 are compared with the oracle in full."""
    skipped = _check(32, 3, 1024, 1024, (8, 16), seed=4, images=[0, 31])
    assert skipped < 0.01 * 2 * 3 * 1024 * 1024


def test_soft_rejects_bad_arguments():
    x = torch.zeros((1, 3, 16, 16), device="cuda")
    w = torch.zeros((1, 1, 16, 16), device="cuda")
    with pytest.raises(P.DppixError):
        P.soft_forward(x, w, P.SoftSpec(grids=(0, 8)))
    with pytest.raises(P.DppixError):
        P.soft_forward(x, w, P.SoftSpec(grids=(8, 256)))
    with pytest.raises(ValueError):
        P.soft_forward(x, torch.zeros((1, 1, 8, 16), device="cuda"), P.SoftSpec())
