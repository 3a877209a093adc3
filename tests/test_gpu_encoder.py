"""Band encoder of the learned band (dtw_encode, dtw_encoder_grad,
dtw_encoder_adam, dtw_align_learned).

The encoder is not part of the exact method: the exact DP inside the band
and the fallback to the full exact DP keep the alignment exact, and the
tests of the band pipeline check exactly that.  The encoder's own kernels
(forward, hand-derived backward, Adam) are compared with a plain PyTorch CPU
reference of the same network in FP64 with autograd."""
import numpy as np
import pytest

import oracle
from paper_2607_15478_gb300 import band_train, synth
from tests._parity import assert_parity, path_tol, total_tol
from tests._pins import check_path_valid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = torch.nn.functional
TAU, WIN, Q, MARGIN, WMIN, WMAX = 0.1, 16, 0.9, 64.0, 256.0, 2048.0


@pytest.fixture(scope="module")
def aligner():
    from paper_2607_15478_gb300 import build, pardtw
    build.build()
    a = pardtw.Aligner(0)
    yield a
    a.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def blocks(p, D):
    lay, _ = band_train.layout(D)
    return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in lay.items()}


def round_bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def ref_forward(X, prm, ds, bf16=False):
    """Pooled, normalised input -> conv5 x3 (relu) -> embedding, width logit,
    half-width (FP64, torch CPU)."""
    X = torch.as_tensor(X, dtype=torch.float64)
    L, D = X.shape
    Lc = (L + ds - 1) // ds
    pooled = torch.stack([X[c * ds:min((c + 1) * ds, L)].mean(0) for c in range(Lc)])
    n = pooled.norm(dim=1, keepdim=True)
    x = torch.where(n > 0, pooled / torch.where(n > 0, n, torch.ones_like(n)), pooled)
    rb = round_bf16 if bf16 else (lambda t: t)
    h = x
    for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        h = torch.relu(F.conv1d(rb(h).T[None], rb(prm[W]), prm[b], padding=2)[0].T)
    z = rb(h) @ rb(prm["W4"]).T + prm["b4"]
    e = z / z.norm(dim=1, keepdim=True)
    s = h @ prm["W5"] + prm["b5"]
    hw = WMIN * (WMAX / WMIN) ** torch.sigmoid(s)
    return e, s, hw, x


def params_t(p, D, grad=False):
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=grad)
         for k, v in blocks(p.astype(np.float64), D).items()}
    return t


@pytest.mark.parametrize("L,ds", [(500, 8), (2003, 8), (96, 4), (1, 8)])
@pytest.mark.parametrize("bf16", [False, True])
def test_encode_matches_reference(aligner, L, ds, bf16):
    rng = np.random.default_rng(L + ds)
    X = synth.chroma_frames(rng, L).astype(np.float32)
    p = band_train.init_params(12, seed=L)
    e_ref, s_ref, hw_ref, _ = ref_forward(X, params_t(p, 12), ds, bf16)
    emb, hw = aligner.encode(dev(X), dev(p), downsample=ds, bf16=bf16)
    tol = 2e-3 if bf16 else 2e-5
    np.testing.assert_allclose(emb.cpu().numpy(), e_ref.numpy(), atol=tol, rtol=0)
    np.testing.assert_allclose(hw.cpu().numpy(), hw_ref.detach().numpy(), rtol=tol * 10)


def targets(path, La, Lb, ds):
    Lac, Lbc = (La + ds - 1) // ds, (Lb + ds - 1) // ds
    s, n = np.zeros(Lac), np.zeros(Lac)
    np.add.at(s, path[:, 0] // ds, path[:, 1])
    np.add.at(n, path[:, 0] // ds, 1)
    return np.minimum((s / n / ds).astype(np.int64), Lbc - 1)


def ref_loss_emb(A, B, prm, ds, tgt):
    eA = ref_forward(A, prm, ds)[0]
    eB = ref_forward(B, prm, ds)[0]
    Lbc = eB.shape[0]
    total = 0.0
    for i, c in enumerate(tgt):
        j0, j1 = max(c - WIN, 0), min(c + WIN, Lbc - 1)
        lg = eB[j0:j1 + 1] @ eA[i] / TAU
        total = total + (torch.logsumexp(lg, 0) - lg[c - j0])
    return total / len(tgt)


@pytest.mark.parametrize("La,Lb", [(800, 950), (1500, 1300)])
def test_embedding_gradient_matches_autograd(aligner, La, Lb):
    wp = synth.warped_pair(synth.rng_for(70, La), La, Lb, 12, knots=8, tmin=0.6, tmax=1.6)
    A, B = dev(wp.A), dev(wp.B)
    path, _ = aligner.align(A, B)
    plen = torch.tensor([path.shape[0]], dtype=torch.int32, device="cuda")
    p = band_train.init_params(12, seed=3)
    P = dev(p)
    G = torch.zeros_like(P)
    loss = torch.zeros(1, device="cuda")
    from paper_2607_15478_gb300 import pardtw
    pardtw.dtw_encoder_grad(aligner.h, P, A, B, path.contiguous(), plen, 0, G, loss)
    torch.cuda.synchronize()
    prm = params_t(p, 12, grad=True)
    tgt = targets(path.cpu().numpy(), La, Lb, 8)
    L = ref_loss_emb(wp.A, wp.B, prm, 8, tgt)
    L.backward()
    assert abs(float(loss.item()) - float(L.detach())) <= 1e-4 * abs(float(L.detach())) + 1e-6
    g = blocks(G.cpu().numpy(), 12)
    for k, t in prm.items():
        if k in ("W5", "b5"):
            assert np.abs(g[k]).max() == 0.0, k  # mode 0 leaves the width head alone
            continue
        ref = t.grad.numpy()
        scale = np.abs(ref).max() + 1e-12
        np.testing.assert_allclose(g[k], ref, atol=2e-4 * scale, rtol=0, err_msg=k)


def test_width_gradient_matches_autograd(aligner):
    La, Lb = 1200, 1400
    wp = synth.warped_pair(synth.rng_for(71, La), La, Lb, 12, knots=8, tmin=0.6, tmax=1.6)
    A, B = dev(wp.A), dev(wp.B)
    path, _ = aligner.align(A, B)
    plen = torch.tensor([path.shape[0]], dtype=torch.int32, device="cuda")
    p = band_train.init_params(12, seed=5)
    P = dev(p)
    G = torch.zeros_like(P)
    loss = torch.zeros(1, device="cuda")
    from paper_2607_15478_gb300 import pardtw
    pardtw.dtw_encoder_grad(aligner.h, P, A, B, path.contiguous(), plen, 1, G, loss)
    # the coarse alignment of the library's own embeddings, as the call makes it
    eA, _ = aligner.encode(A, P)
    eB, _ = aligner.encode(B, P)
    cpath, _ = aligner.align(eA, eB)
    cp, fp = cpath.cpu().numpy(), path.cpu().numpy()
    Lac = eA.shape[0]
    need = np.zeros(Lac)
    for i in range(Lac):
        sel = (cp[:, 0] >= i - 1) & (cp[:, 0] <= i + 1)
        f0, f1 = cp[sel, 1].min() * 8, (cp[sel, 1].max() + 1) * 8 - 1
        js = fp[(fp[:, 0] >= 8 * i) & (fp[:, 0] < 8 * i + 8), 1]
        need[i] = max(0, (f0 - js).max(), (js - f1).max())
    wt = np.clip(np.log2((need + MARGIN) / WMIN) / np.log2(WMAX / WMIN), 0, 1)
    prm = params_t(p, 12, grad=True)
    s = ref_forward(wp.A, prm, 8)[1]
    d = torch.tensor(wt) - torch.sigmoid(s)
    L = torch.where(d > 0, Q * d, (Q - 1) * d).mean()
    L.backward()
    torch.cuda.synchronize()
    assert abs(float(loss.item()) - float(L.detach())) <= 1e-4 * abs(float(L.detach())) + 1e-6
    g = blocks(G.cpu().numpy(), 12)
    for k, t in prm.items():
        if k in ("W5", "b5"):
            ref = t.grad.numpy()
            np.testing.assert_allclose(g[k], ref, atol=2e-4 * (np.abs(ref).max() + 1e-12),
                                       rtol=0, err_msg=k)
        else:
            assert np.abs(g[k]).max() == 0.0, k  # mode 1 leaves the trunk alone


def test_adam_step(aligner):
    from paper_2607_15478_gb300 import pardtw
    rng = np.random.default_rng(9)
    p, g = rng.standard_normal(1000), rng.standard_normal(1000)
    m, v = rng.standard_normal(1000) * 0.1, rng.random(1000) * 0.1
    P, G, M, V = dev(p), dev(g), dev(m), dev(v)
    pardtw.dtw_encoder_adam(aligner.h, P, G, M, V, 3, 0.01)
    torch.cuda.synchronize()
    m1 = 0.9 * m + 0.1 * g
    v1 = 0.999 * v + 0.001 * g * g
    p1 = p - 0.01 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    np.testing.assert_allclose(P.cpu().numpy(), p1, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(M.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    assert float(G.abs().max()) == 0.0


def test_training_reduces_loss(aligner):
    from paper_2607_15478_gb300 import pardtw
    pairs = [synth.band_training_pair(k, La=1500) for k in range(6)]
    As = [dev(q.A) for q in pairs]
    Bs = [dev(q.B) for q in pairs]
    paths, lens = band_train.exact_paths(aligner, As, Bs)
    P = dev(band_train.init_params(12, seed=1))
    G, M, V = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
    loss = torch.zeros(1, device="cuda")
    hist, step = [], 0
    for ep in range(8):
        loss.zero_()
        for k in range(len(pairs)):
            pardtw.dtw_encoder_grad(aligner.h, P, As[k], Bs[k], paths[k], lens[k], 0, G, loss)
            step += 1
            pardtw.dtw_encoder_adam(aligner.h, P, G, M, V, step, 3e-3)
        hist.append(float(loss.item()) / len(pairs))
    assert hist[-1] < 0.7 * hist[0], hist


@pytest.mark.parametrize("La,Lb", [(300, 360), (1000, 1200), (2500, 2000), (4000, 5000)])
def test_learned_band_is_exact_or_falls_back(aligner, La, Lb):
    # untrained weights: the band is what it is; the result is the exact
    # alignment (judged by the FP64 oracle) whenever the exact path lies
    # inside the band or the fallback ran; otherwise the optimum inside the
    # band, never below the exact optimum
    wp = synth.warped_pair(synth.rng_for(72, La), La, Lb, 12, knots=16, tmin=0.6, tmax=1.6)
    A, B = dev(wp.A), dev(wp.B)
    P = dev(band_train.init_params(12, seed=2))
    po, to = oracle.dtw(wp.A, wp.B)
    for bf16 in (False, True):
        path, total, fb = aligner.align_learned(A, B, P, bf16=bf16)
        p = path.cpu().numpy()
        check_path_valid(p, La, Lb)
        tg = oracle.path_cost(wp.A, wp.B, p)
        if fb or tg - to <= path_tol(to, La, Lb):
            assert_parity(wp.A, wp.B, p, total, name="learned-band", ref=(po, to))
        else:
            assert abs(total - tg) <= total_tol(tg, La, Lb)
            cells = aligner.band_cells()
            assert 0 < cells <= ((La + 92) // 93) * 93 * Lb


def test_learned_band_trained_multi_wave_matches_oracle(aligner):
    # the trained encoder on the learned-band workload's recipe (tempo 0.6-1.6,
    # 256 knots per 1e5 frames) at 30000 x 36000: the band's sweep has 387
    # strips in 194 groups, several waves of CTAs; the result must be DTW's
    # exact path without a fallback
    La, Lb = 30000, 36000
    wp = synth.warped_pair(synth.rng_for(73, La), La, Lb, 12, knots=77, tmin=0.6, tmax=1.6)
    P = band_train.load(device="cuda")
    for bf16 in (True, False):
        path, total, fb = aligner.align_learned(dev(wp.A), dev(wp.B), P, bf16=bf16)
        assert not fb
        assert 0 < aligner.band_cells() < 0.1 * La * Lb
        ref = assert_parity(wp.A, wp.B, path, total, name="learned-band-multi-wave",
                            ref=None if bf16 else ref)


def test_band_cells_of_banded_call(aligner):
    wp = synth.config_pair(0)
    A, B = dev(wp.A), dev(wp.B)
    path, total, fb = aligner.align_banded(A, B, downsample=8, halfwidth=32)
    assert not fb
    cells = aligner.band_cells()
    assert 0 < cells < wp.A.shape[0] * wp.B.shape[0]
