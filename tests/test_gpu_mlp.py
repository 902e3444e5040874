"""The tensor-core surrogate MLP against torch and the FP64 oracle (needs a
GB300)."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2311_15088_gb300 import sph

pytestmark = pytest.mark.gpu


def _bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16)


@pytest.mark.parametrize("grad", [0, 1, 2])
def test_gelu_against_exact_erf(grad):
    """The kernels' GELU (erf by Abramowitz and Stegun 7.1.26 in float32;
    grad = 2 the packed two-value form of the fused forward) against the
    exact-erf GELU in float64, over a dense grid of inputs covering the range
    the network's pre-activations take and beyond."""
    import math

    z = np.concatenate([np.linspace(-12.0, 12.0, 200001), [0.0, -0.0, 1e-30, -1e-30, 40.0, -40.0]]).astype(np.float32)
    zd = torch.from_numpy(z).cuda()
    out = torch.empty_like(zd)
    sph.sph_debug_gelu(zd.data_ptr(), len(z), grad, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = out.cpu().double().numpy()
    zz = z.astype(np.float64)
    phi = np.array([0.5 * (1.0 + math.erf(v / math.sqrt(2.0))) for v in zz])
    ref = zz * phi if grad != 1 else phi + zz * np.exp(-0.5 * zz * zz) / math.sqrt(2.0 * math.pi)
    # |erf error| <= 1.5e-7 (the formula) plus float32 evaluation: 1e-6
    # absolute on Phi, times |z| for GELU
    tol = 1e-6 * np.maximum(1.0, np.abs(zz)) + 1e-6 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))


@pytest.mark.parametrize("M,N,K,splits", [(128, 256, 272, 1), (300, 16, 256, 1), (256, 272, 1024, 4),
                                          (16, 256, 4096, 8), (384, 128, 64, 1), (130, 256, 16, 1)])
def test_tcgen05_gemm_matches_fp32_product(M, N, K, splits):
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((splits, M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(4, dtype=torch.int32, device="cuda")
    kb = (K + 63) // 64
    s = min(splits, kb)
    per = (kb + s - 1) // s
    s = (kb + per - 1) // per
    sph.sph_debug_gemm(A.data_ptr(), K, B.data_ptr(), K, M, N, K, splits, C.data_ptr(), err.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(err[0]) == 0
    got = C[:s].sum(0).double()
    ref = A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T)
    assert torch.all((got - ref).abs() <= 1e-5 * scale + 1e-6), float(((got - ref).abs() / scale).max())


def _oracle_params_bf16(seed):
    """Oracle parameters with the weights rounded to BF16 (what the tensor
    cores see) and small random biases."""
    p = omlp.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for w, b, n_out, _ in omlp.LAYERS:
        p[w] = _bf16(p[w]).double().numpy()
        p[b] = rng.uniform(-0.1, 0.1, size=n_out)
    return p


def _pack(p):
    return np.concatenate([np.concatenate([p[w].ravel(), p[b]]) for w, b, _, _ in omlp.LAYERS]).astype(np.float32)


def _unpack(v):
    out, o = {}, 0
    for w, b, n_out, n_in in omlp.LAYERS:
        out[w] = v[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        out[b] = v[o:o + n_out]
        o += n_out
    return out


def _inputs(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, omlp.D_IN))
    x[:, 259:] = 0
    return _bf16(x).double().numpy()


def test_forward_matches_oracle():
    p = _oracle_params_bf16(11)
    x = _inputs(640, 12)
    m = sph.Mlp(1024)
    m.set_params(torch.from_numpy(_pack(p)))
    y = m.forward(_bf16(x).cuda()).double().cpu().numpy()
    assert m.status() == 0
    ref = omlp.forward(p, x)["y"]
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel <= 2e-2, rel
    assert np.all(np.abs(y - ref) <= 2e-2 * np.abs(ref).max())


@pytest.mark.parametrize("tiles", [153, 305, 512])
def test_forward_many_tiles_matches_oracle(tiles):
    """The fused forward with more 128-row tiles than SMs (each CTA loops
    over several tiles, the last ones ragged across CTAs): a sample of rows
    from every tile against the oracle, and the whole batch against the
    same rows run as a batch of their own (tile placement changes nothing)."""
    B = 128 * tiles
    p = _oracle_params_bf16(31)
    x = _inputs(B, 32)
    m = sph.Mlp(B)
    m.set_params(torch.from_numpy(_pack(p)))
    xb = _bf16(x).cuda()
    y = m.forward(xb).double().cpu().numpy()
    assert m.status() == 0
    rows = np.arange(5, B, 29)
    assert len(np.unique(rows // 128)) == tiles
    ref = omlp.forward(p, x[rows])["y"]
    assert np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref) <= 2e-2
    assert np.all(np.abs(y[rows] - ref) <= 2e-2 * np.abs(ref).max())
    # the last 640 rows as a batch of their own: bit-identical outputs
    y2 = m.forward(xb[-640:]).cpu().numpy()
    assert np.array_equal(y2, y[-640:].astype(np.float32))


def test_gradients_match_oracle():
    p = _oracle_params_bf16(21)
    x = _inputs(512, 22)
    rng = np.random.default_rng(23)
    dy = np.zeros((512, omlp.D_OUT))
    dy[:, :4] = rng.normal(size=(512, 4)) / 512
    m = sph.Mlp(512)
    m.set_params(torch.from_numpy(_pack(p)))
    g = m.gradients(_bf16(x).cuda(), torch.from_numpy(dy.astype(np.float32)).cuda()).double().cpu().numpy()
    assert m.status() == 0
    ref = omlp.backward(p, omlp.forward(p, x), dy)
    got = _unpack(g)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        a, b = got[name].ravel(), ref[name].ravel()
        if name in ("W4", "b4"):
            a, b = got[name][:4].ravel(), ref[name][:4].ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert cos >= 0.999, (name, cos)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(5)
    B = 4096
    x = rng.normal(size=(B, omlp.D_IN)) * 0.5
    x[:, 259:] = 0
    t = np.zeros((B, 4))
    t[:, 0] = np.tanh(x[:, 0] + 0.5 * x[:, 1])
    t[:, 1] = x[:, 2] * x[:, 3]
    t[:, 2] = np.sin(x[:, 4])
    m = sph.Mlp(B)
    m.set_params(torch.from_numpy(_pack(omlp.init_params(6))))
    xb = _bf16(x).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    first = None
    for it in range(300):
        loss = float(m.train_step(xb, tt, 1e-3).item()) if it % 50 == 0 or it == 299 else m.train_step(xb, tt, 1e-3)
        if it == 0:
            first = loss
    last = float(m.loss.item())
    assert m.status() == 0
    assert last < 0.2 * first, (first, last)
    # the GPU forward of the trained weights agrees with the oracle forward
    pt = m.get_params().double().cpu().numpy()
    q = _unpack(pt)
    for w, _, _, _ in omlp.LAYERS:
        q[w] = _bf16(q[w]).double().numpy()
    y = m.forward(xb[:512]).double().cpu().numpy()
    ref = omlp.forward(q, _bf16(x[:512]).double().numpy())["y"]
    assert np.linalg.norm(y[:, :3] - ref[:, :3]) / np.linalg.norm(ref[:, :3]) <= 3e-2


def _flat(d):
    return np.concatenate([np.concatenate([d[w].ravel(), d[b].ravel()]) for w, b, _, _ in omlp.LAYERS])


def _trained_blocks(phase):
    """(name, index array into the packed parameters) of what a phase trains:
    phase 0 every parameter but the error head (row 3 of W4, b4[3]), phase 1
    the error head only; rows 4..15 of W4 and b4[4..15] (padding outputs)
    have zero gradient and are left out of the comparison of directions."""
    idx, o = {}, 0
    for w, b, n_out, n_in in omlp.LAYERS:
        W = o + np.arange(n_out * n_in).reshape(n_out, n_in)
        o += n_out * n_in
        bb = o + np.arange(n_out)
        o += n_out
        if w == "W4":
            if phase == 0:
                idx["W4[0:3]"], idx["b4[0:3]"] = W[:3].ravel(), bb[:3]
            else:
                idx["W4[3]"], idx["b4[3]"] = W[3], bb[3:4]
        elif phase == 0:
            idx[w], idx[b] = W.ravel(), bb
    trained = np.zeros(o, bool)
    if phase == 0:
        trained[:] = True
        trained[idx_row3(o)] = False
    else:
        trained[np.concatenate(list(idx.values()))] = True
    return idx, trained


def idx_row3(total):
    """Packed indices of the error head: row 3 of W4 and b4[3]."""
    o = sum(n_out * n_in + n_out for _, _, n_out, n_in in omlp.LAYERS[:3])
    w4 = o + 3 * omlp.D_H + np.arange(omlp.D_H)
    b4 = o + omlp.D_OUT * omlp.D_H + 3
    return np.concatenate([w4, [b4]])


@pytest.mark.parametrize("phase", [0, 1])
def test_train_steps_match_oracle_adam(phase):
    """Three sph_mlp_train_step calls from fixed parameters and batch, each
    checked against the FP64 oracle: (1) the step's gradient against the
    oracle's gradient of the BF16-rounded network at the step's starting
    weights (cosine >= 0.999 per block, the BF16 bound of
    test_gradients_match_oracle), (2) the Adam update (first and second
    moments and the FP32 master weights) element by element against the
    oracle's adam_update applied to that gradient, within the float32
    rounding of the kernel's operations, (3) every parameter the phase does
    not train left bit for bit unchanged, (4) the loss within BF16 accuracy."""
    B, lr = 512, 2e-3
    p = _oracle_params_bf16(41)
    x = _inputs(B, 42)
    rng = np.random.default_rng(43)
    t = rng.normal(size=(B, 4))
    t[:, 3] = rng.uniform(-3, 0, size=B)
    m = sph.Mlp(B)
    m.set_params(torch.from_numpy(_pack(p)))
    xb = _bf16(x).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    b1, b2, eps = (float(np.float32(v)) for v in (0.9, 0.999, 1e-8))
    blocks, trained = _trained_blocks(phase)
    w_prev = m.get_params().double().cpu().numpy()
    m_prev = np.zeros_like(w_prev)
    v_prev = np.zeros_like(w_prev)
    for step in (1, 2, 3):
        loss = float(m.train_step(xb, tt, lr, phase).item())
        g, m1, m2, k = m.optimizer_state()
        g, m1, m2 = (a.double().cpu().numpy() for a in (g, m1, m2))
        w = m.get_params().double().cpu().numpy()
        assert k == step and m.status() == 0
        # (1) the gradient against the oracle's of the BF16-rounded network
        q = _unpack(w_prev)
        for name, _, _, _ in omlp.LAYERS:
            q[name] = _bf16(q[name]).double().numpy()
        c = omlp.forward(q, x)
        if phase == 0:
            dy, lref = omlp.force_loss_grad_y(c["y"], t[:, :3]), omlp.force_loss(c["y"], t[:, :3])
        else:
            dy = omlp.error_loss_grad_y(c["y"], t[:, 3])
            lref = 0.5 * float(np.sum((c["y"][:, 3] - t[:, 3]) ** 2)) / B
        gref = _flat(omlp.backward(q, c, dy))
        for name, ix in blocks.items():
            a, b = g[ix], gref[ix]
            cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
            assert cos >= 0.999, (step, name, cos)
        assert abs(loss - lref) <= 2e-2 * lref, (loss, lref)
        # (2) Adam on the GPU's gradient, element by element
        wr, mr, vr = omlp.adam_update(w_prev, g, m_prev, v_prev, step, lr, b1, b2, eps)
        tr = trained
        assert np.all(np.abs(m1[tr] - mr[tr]) <= 3e-7 * (b1 * np.abs(m_prev[tr]) + (1 - b1) * np.abs(g[tr])) + 1e-38)
        assert np.all(np.abs(m2[tr] - vr[tr]) <= 4e-7 * (b2 * v_prev[tr] + (1 - b2) * g[tr] ** 2) + 1e-38)
        upd = np.abs(wr - w_prev)
        # the update's error: the first moment's (it can cancel, so its
        # error is relative to its terms, not to itself) carried through
        # lr / (sqrt(v_hat) + eps), a few float32 roundings of the update,
        # and the rounding of the new weight
        dm = 3e-7 * (b1 * np.abs(m_prev) + (1 - b1) * np.abs(g)) / (1 - b1 ** step)
        tol_w = lr * dm / (np.sqrt(vr / (1 - b2 ** step)) + eps) + 2e-6 * upd + 6e-8 * np.abs(wr) + 1e-38
        bad = np.nonzero(tr & (np.abs(w - wr) > tol_w))[0]
        assert len(bad) == 0, (step, len(bad), [(int(i), g[i], m1[i], m2[i], w_prev[i], w[i], wr[i]) for i in bad[:6]])
        # the update moved the trained parameters by about lr
        assert 0.3 * lr < np.median(upd[tr][np.abs(g[tr]) > 1e-6]) < 3.0 * lr
        # (3) untouched parameters and moments
        assert np.array_equal(w[~tr], w_prev[~tr])
        assert np.array_equal(m1[~tr], m_prev[~tr]) and np.array_equal(m2[~tr], v_prev[~tr])
        w_prev, m_prev, v_prev = w, m1, m2


def test_checkpoint_resumes_training_bit_for_bit(tmp_path):
    """Two Adam steps, a checkpoint (state_dict through torch.save), two more
    steps; a fresh network loaded from the checkpoint takes the same two
    steps: parameters and both moments bit for bit equal."""
    B, lr = 256, 1e-3
    x = _bf16(_inputs(B, 52)).cuda()
    rng = np.random.default_rng(53)
    t = torch.from_numpy(rng.normal(size=(B, 4)).astype(np.float32)).cuda()
    a = sph.Mlp(B)
    a.set_params(torch.from_numpy(_pack(_oracle_params_bf16(51))))
    for _ in range(2):
        a.train_step(x, t, lr)
    path = tmp_path / "mlp.pt"
    torch.save({k: v.cpu() for k, v in a.state_dict().items()}, path)
    for _ in range(2):
        a.train_step(x, t, lr)
    b = sph.Mlp(B)
    b.load_state_dict(torch.load(path))
    for _ in range(2):
        b.train_step(x, t, lr)
    sa, sb = a.state_dict(), b.state_dict()
    assert int(sa["adam_step"]) == int(sb["adam_step"]) == 4
    for k in ("params", "adam_m1", "adam_m2"):
        assert torch.equal(sa[k], sb[k]), k
    assert a.status() == 0 and b.status() == 0
