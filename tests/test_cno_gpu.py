"""GPU parity of the surrogate's tensor-core kernels with the FP64 reference
(oracle/cno.py): single convolutions (forward, data gradient, weight
gradient) element by element, then the whole network's output and
per-layer gradients, the Adam update, and a short fit.

The kernels take BF16 operands and accumulate in FP32.  The reference is fed
the same BF16 values and computes in FP64, so the bars are:
  BF16 outputs: |gpu - ref| <= 2^-8 |ref| + 2^-12 sum|terms|  (one rounding to
  8 significant bits, plus FP32 accumulation of up to 2304 products);
  FP32 outputs (weight gradients over many pixels): <= 2^-13 sum|terms|.
Through the whole network every activation and gradient is rounded to BF16,
so the network is compared in relative L2 norm (bars stated in the tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cno as R  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09422_gb300 import _build
    _build.build()
    from paper_2511_09422_gb300 import cno
    cno.load()
    cno.read_status(clear=True)
    yield
    assert cno.read_status() == 0, "a tensor-core kernel gave up a wait"


def _bf16(a, dev="cuda"):
    """(device bf16 tensor, the same values as float64 numpy)."""
    t = torch.as_tensor(np.asarray(a, np.float32)).to(dev).to(torch.bfloat16)
    return t, t.float().cpu().double().numpy()


def _np(t):
    return t.float().cpu().double().numpy()


def _check_bf16_out(got, ref, ref_abs, what):
    tol = 2.0 ** -8 * np.abs(ref) + 2.0 ** -12 * ref_abs + 1e-30
    bad = np.abs(got - ref) > tol
    assert not bad.any(), "%s: %d of %d outside the bar, worst excess %.3e" % (
        what, int(bad.sum()), bad.size, float((np.abs(got - ref) - tol).max()))


FWD_CASES = [
    # n, h, w, cin, cout, act, f32 head
    (2, 8, 8, 64, 64, True, False),       # w < 128: 8 x 16 tiles, rows beyond h masked
    (1, 5, 160, 128, 128, True, False),   # ragged tile in w (128 + 32) and in h
    (1, 3, 256, 64, 256, False, False),   # 256 output channels, no activation
    (2, 16, 32, 256, 64, True, False),    # 256 input channels (4 K blocks per tap)
    (1, 16, 128, 64, 64, False, True),    # FP32 head output, first 8 channels
]


@pytest.mark.parametrize("n,h,w,cin,cout,act,f32", FWD_CASES)
def test_conv_forward_matches_reference(n, h, w, cin, cout, act, f32):
    from paper_2511_09422_gb300 import cno
    rng = np.random.default_rng(11 + cin + cout + h)
    x, xr = _bf16(rng.standard_normal((n, h, w, cin)))
    wt, wr = _bf16(rng.standard_normal((cout, 9, cin)) / np.sqrt(9 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    bt = torch.as_tensor(b).cuda()
    y = cno.conv3x3_forward(x, wt, bt, act, out_f32=f32, n_store=8 if f32 else None)
    torch.cuda.synchronize()
    z = R.conv3x3(xr, wr, b.astype(np.float64))
    ref = R.lrelu(z) if act else z
    ref_abs = R.conv3x3(np.abs(xr), np.abs(wr), np.abs(b.astype(np.float64)))
    if f32:
        got = y.cpu().double().numpy()
        ref, ref_abs = ref[..., :8], ref_abs[..., :8]
        assert np.all(np.abs(got - ref) <= 2.0 ** -12 * ref_abs + 1e-30)
    else:
        _check_bf16_out(_np(y), ref, ref_abs, "forward")


@pytest.mark.parametrize("n,h,w,cout,cin,slope", [(2, 16, 32, 128, 64, True), (1, 8, 256, 64, 256, False),
                                                   (1, 4, 4, 256, 256, True)])
def test_conv_dgrad_matches_reference(n, h, w, cout, cin, slope):
    from paper_2511_09422_gb300 import cno
    rng = np.random.default_rng(21 + cin + cout)
    dz, dzr = _bf16(rng.standard_normal((n, h, w, cout)))
    w32 = (rng.standard_normal((cout, 9, cin)) / np.sqrt(9 * cout)).astype(np.float32)
    wf, wd = cno.weights_to_bf16(torch.as_tensor(w32).cuda())
    wr = _np(wf)
    # the data-gradient matrix is the forward matrix with taps reversed and transposed
    assert np.array_equal(_np(wd), wr[:, ::-1, :].transpose(2, 1, 0))
    y, yr = _bf16(rng.standard_normal((n, h, w, cin))) if slope else (None, None)
    dx = cno.conv3x3_dgrad(dz, wd, y)
    torch.cuda.synchronize()
    xdummy = np.zeros((n, h, w, cin))
    ref, _, _ = R.conv3x3_backward(xdummy, wr, dzr)
    ref_abs, _, _ = R.conv3x3_backward(xdummy, np.abs(wr), np.abs(dzr))
    if slope:
        s = R.lrelu_slope(yr)
        ref, ref_abs = ref * s, ref_abs * s
    _check_bf16_out(_np(dx), ref, ref_abs, "dgrad")


@pytest.mark.parametrize("n,h,w,cin,cout", [(2, 16, 16, 64, 64), (1, 32, 128, 128, 256), (1, 8, 8, 256, 128),
                                            (3, 24, 64, 64, 128)])
def test_conv_wgrad_matches_reference(n, h, w, cin, cout):
    from paper_2511_09422_gb300 import cno
    rng = np.random.default_rng(31 + cin + cout + n)
    dz, dzr = _bf16(rng.standard_normal((n, h, w, cout)))
    x, xr = _bf16(rng.standard_normal((n, h, w, cin)))
    dw, db = cno.conv3x3_wgrad(dz, x)
    torch.cuda.synchronize()
    _, ref_w, ref_b = R.conv3x3_backward(xr, np.zeros((cout, 9, cin)), dzr)
    _, abs_w, abs_b = R.conv3x3_backward(np.abs(xr), np.zeros((cout, 9, cin)), np.abs(dzr))
    got_w = dw.cpu().double().numpy()
    got_b = db.cpu().double().numpy()
    assert np.all(np.abs(got_w - ref_w) <= 2.0 ** -13 * abs_w + 1e-30), float(np.abs(got_w - ref_w).max())
    assert np.all(np.abs(got_b - ref_b) <= 2.0 ** -13 * abs_b + 1e-30)


def _random_params(rng, shapes):
    out = []
    for ci, co in shapes:
        out.append(((rng.standard_normal((co, 9, ci)) * np.sqrt(2.0 / (9 * ci))).astype(np.float32),
                    (0.1 * rng.standard_normal(co)).astype(np.float32)))
    return out


def _net_case(seed=41, n=2, h=32, w=32):
    from paper_2511_09422_gb300 import cno
    rng = np.random.default_rng(seed)
    params = _random_params(rng, cno.layer_shapes())
    xin = np.zeros((n, h, w, cno.CIN), np.float32)
    xin[..., :cno.NF] = rng.standard_normal((n, h, w, cno.NF))
    target = rng.standard_normal((n, h, w, cno.NF)).astype(np.float32)
    return params, xin, target


def _bf16_params(params):
    """The values the tensor cores see: BF16 weights, FP32 biases."""
    return [(torch.as_tensor(w).to(torch.bfloat16).double().numpy(), b.astype(np.float64)) for w, b in params]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_network_forward_and_gradients_match_reference():
    from paper_2511_09422_gb300 import cno
    params, xin, target = _net_case()
    net = cno.Net()
    net.set_params(cno.flatten(params))
    x, xr = _bf16(xin)
    tt = torch.as_tensor(target).cuda()
    loss = net.train_step(x, tt, lr=0.0, update=False)
    out_gpu = net.forward(x).cpu().double().numpy()
    grads = cno.unflatten(net.grads())
    p64 = _bf16_params(params)
    out_ref, cache = R.forward(p64, xr)
    loss_ref, dout = R.mse(out_ref, np.concatenate([target, np.zeros(target.shape[:3] + (cno.COUT - cno.NF,))],
                                                    axis=-1).astype(np.float64), cno.NF)
    g_ref = R.backward(p64, cache, dout)
    e_out = _rel(out_gpu, out_ref[..., :cno.NF])
    assert e_out <= 1e-2, e_out
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref, (loss, loss_ref)
    errs = []
    for k in range(12):
        ew = _rel(grads[k][0].astype(np.float64), g_ref[k][0])
        eb = _rel(grads[k][1].astype(np.float64), g_ref[k][1])
        errs.append((k, ew, eb))
    # BF16 activations and gradients through up to 12 layers: 5 % in norm
    assert all(ew <= 5e-2 and eb <= 5e-2 for _, ew, eb in errs), errs
    net.close()


def test_adam_update_matches_reference():
    from paper_2511_09422_gb300 import cno
    params, xin, target = _net_case(seed=43, n=1, h=16, w=16)
    net = cno.Net()
    flat0 = cno.flatten(params)
    net.set_params(flat0)
    x, _ = _bf16(xin)
    tt = torch.as_tensor(target).cuda()
    lr = 1e-3
    net.train_step(x, tt, lr=lr, update=True)
    g = net.grads().astype(np.float64)
    p1 = net.params().astype(np.float64)
    want, m, v = R.adam(flat0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    assert np.all(np.abs(p1 - want) <= 1e-6 * lr + 2.0 ** -22 * np.abs(want)), float(np.abs(p1 - want).max())
    net.close()


def test_training_reduces_loss_on_a_fixed_batch():
    from paper_2511_09422_gb300 import cno
    params, xin, _ = _net_case(seed=47, n=4, h=32, w=32)
    # a learnable target: a smooth function of the input fields
    target = np.tanh(xin[..., :cno.NF] * 0.5).astype(np.float32)
    net = cno.Net()
    net.set_params(cno.flatten(params))
    x, _ = _bf16(xin)
    tt = torch.as_tensor(target).cuda()
    first = net.train_step(x, tt, lr=1e-3)
    for _ in range(60):
        last = net.train_step(x, tt, lr=1e-3, want_loss=False)
    last = net.train_step(x, tt, lr=1e-3, update=False)
    assert last < 0.2 * first, (first, last)
    net.close()


def test_bounded_wait_gives_up_and_reports():
    """Failure detection without a GPU fault: the barrier wait every tensor-core
    kernel uses gives up after its limit on a barrier that nothing arrives at,
    and the device stays usable."""
    from paper_2511_09422_gb300 import cno
    gave_up, elapsed = cno.wait_selftest(0.2)
    assert gave_up
    assert 0.2 <= elapsed <= 2.0, elapsed
    x = torch.zeros(4, device="cuda") + 1.0   # the context is still usable
    assert float(x.sum()) == 4.0
    assert cno.read_status() == 0
