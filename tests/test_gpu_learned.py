"""Learned correction on the GPU: the library's BF16/FP32 MLP kernels against
the FP64 reference (oracle/learned.py), training on oracle-generated
(features, exact cardinality) pairs, and the gain over the plain estimate on
held-out seeds.

Training data: trace-shaped runs (Zipf 1.05, 10% in-slice repeats, k = 30,
g = 256, 31 slices) at 1/32 of the trace's pairs, hosts, top cardinality and
pool, seeds 1000..1007; evaluation seed 0 (disjoint).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import exact, learned  # noqa: E402
from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15
SCALE = 32


@pytest.fixture(scope="module")
def data():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Xtr, ptr, ctr = learned.training_set(range(1000, 1008), scale=SCALE, processes=8)
    Xev, pev, cev = learned.trace_shaped_run(0, scale=SCALE)
    torch.cuda.set_device(0)
    return Xtr, ptr, ctr, Xev, pev, cev


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def _dev_live(X80):
    from paper_1810_13132_gb300 import live_features
    return _bf16(live_features(X80)).cuda()


def _rounded_reference_params(params):
    """The parameters as the GPU sees them: W1, W2 in BF16, the rest FP32."""
    p = params.astype(np.float64).copy()
    for name in ("W1", "W2"):
        off, k = 0, 0
        for n, shape in learned.SIZES:
            if n == name:
                k = int(np.prod(shape))
                break
            off += int(np.prod(shape))
        p[off:off + k] = _bf16(p[off:off + k]).float().numpy()
    return p


def _target(n_plain, card):
    return np.log1p(card) - np.log1p(n_plain)


def test_gradient_matches_fp64_reference(data):
    """Every gradient element against the FP64 reference at the parameters
    and inputs the GPU reads (BF16 W1, W2 and X).  The GPU stores h1, dZ2 and
    dZ1 in BF16 (relative rounding 2^-9) and evaluates GELU with the
    hardware tanh (relative error 2^-11), so each term of a gradient sum
    carries a relative error of a few 1e-3; the bound per element is
    2e-2 max(|g_ref|, rms of that layer's gradient), the floor covering
    elements whose terms cancel."""
    from paper_1810_13132_gb300 import Mlp
    Xtr, ptr, ctr = data[:3]
    X, y = Xtr[:1000], _target(ptr[:1000], ctr[:1000])
    m = Mlp(seed=3)
    params, _ = m.get_params()
    params[-1] = 0.1
    m.set_params(params)
    g_gpu, loss_gpu = m.gradient(_dev_live(X), torch.from_numpy(y.astype(np.float32)).cuda())
    Xr = _bf16(X).double().numpy()  # the BF16 inputs the GPU reads
    theta = _rounded_reference_params(params)
    g_ref = learned.gradient(theta, Xr, y)
    assert loss_gpu == pytest.approx(learned.loss(theta, Xr, y), rel=2e-2)
    off = 0
    for name, shape in learned.SIZES:
        k = int(np.prod(shape))
        got, want = g_gpu[off:off + k].astype(np.float64), g_ref[off:off + k]
        live = np.ones(k, bool)
        if name == "W1":
            dead = np.zeros((64, 80), bool)
            dead[:, 32:64] = True  # columns of always-zero inputs: no gradient on either side
            live = ~dead.ravel()
            assert np.abs(got[~live]).max() == 0.0
        rms = np.sqrt(np.mean(want[live] ** 2))
        bound = 2e-2 * np.maximum(np.abs(want[live]), rms)
        ratio = np.abs(got[live] - want[live]) / bound
        worst = int(np.argmax(ratio))
        assert ratio.max() <= 1.0, (name, float(ratio.max()), worst, got[live][worst],
                                    want[live][worst], rms)
        off += k
    assert off == learned.N_PARAMS


def test_forward_matches_fp64_reference(data):
    from paper_1810_13132_gb300 import Mlp
    X = data[0][:3000]
    m = Mlp(seed=4)
    params, _ = m.get_params()
    d_gpu = m.forward(_dev_live(X)).cpu().numpy()
    d_ref, _ = learned.forward(_rounded_reference_params(params), _bf16(X).double().numpy())
    assert np.abs(d_gpu - d_ref).max() < 2e-2 * max(1.0, np.abs(d_ref).max())


def _replay_on_gpu(seed):
    """The evaluation run's traffic through the library: (handle, aips, exact)."""
    from paper_1810_13132_gb300 import Config, Vbdr
    k = 30
    gen = traffic.ZipfTraffic(1_000_000 // SCALE, 1.05, 2_000_000 // SCALE, k, seed=seed,
                              repeat_frac=0.10)
    v = Vbdr(Config(k=k, num_bdr=(1 << 24) // SCALE, log2_g=8, seed=SEED))
    hist = []
    for _ in range(k + 1):
        s = gen.next_slice((64 << 20) // SCALE)
        hist.append(s)
        v.scan(torch.from_numpy(s.view(np.int32)).cuda())
        v.slide()
    truth = exact.window_cardinalities(hist, k, k, gen.aips).astype(np.float64)
    return v, gen.aips, truth


def test_training_gain_and_fused_estimate(data):
    from paper_1810_13132_gb300 import Mlp
    Xtr, ptr, ctr, Xev, pev, cev = data
    perm = np.random.default_rng(0).permutation(ctr.size)
    Xd = _dev_live(Xtr[perm])
    yd = torch.from_numpy(_target(ptr, ctr)[perm].astype(np.float32)).cuda()
    m = Mlp(seed=7)
    losses = m.train(Xd, yd, epochs=40, batch=2048, lr=2e-3, weight_decay=1e-4)
    assert losses[-1] < 0.5 * losses[0], losses
    params, _ = m.get_params()
    nmax = float(ptr.max())
    m.set_params(params, nmax)

    # held-out seed, features from the oracle: corrected vs plain
    delta = m.forward(_dev_live(Xev)).cpu().numpy().astype(np.float64)
    corr = np.where(pev > nmax, pev, learned.correct(pev, delta))
    mre_plain = np.mean(np.abs(pev - cev) / cev)
    mre_corr = np.mean(np.abs(corr - cev) / cev)
    assert mre_corr < 0.6 * mre_plain, (mre_corr, mre_plain)

    # the same traffic through the library: features and the fused estimate
    v, aips, truth = _replay_on_gpu(0)
    live = truth > 0
    d_aips = torch.from_numpy(aips.view(np.int32)).cuda()
    X_gpu, plain_gpu = v.features(d_aips)
    plain = v.estimate(d_aips)
    assert torch.equal(plain_gpu, plain)
    # GPU features equal the oracle's, rounded to BF16
    from paper_1810_13132_gb300 import live_features
    Xo = torch.from_numpy(live_features(Xev).astype(np.float32)).to(torch.bfloat16)
    Xg = X_gpu.cpu()[torch.from_numpy(live)]
    assert torch.equal(Xg[:, :32], Xo[:, :32])  # histogram bins exact
    rel = (Xg[:, 32:38].float() - Xo[:, 32:38].float()).abs() / Xo[:, 32:38].float().abs().clamp_min(1e-3)
    assert rel.max().item() <= 2 ** -7
    fused = v.estimate_learned(m, d_aips).cpu().numpy().astype(np.float64)
    sep = m.forward(X_gpu).cpu().numpy().astype(np.float64)
    p = plain.cpu().numpy().astype(np.float64)
    sep = np.where(p > nmax, p, learned.correct(p, sep))
    np.testing.assert_allclose(fused, sep, rtol=1e-5, atol=1e-3)
    mre_f = np.mean(np.abs(fused[live] - truth[live]) / truth[live])
    mre_p = np.mean(np.abs(p[live] - truth[live]) / truth[live])
    assert mre_f < 0.6 * mre_p, (mre_f, mre_p)


def test_feature_calls_check_alignment_and_g():
    """The feature rows are written with 8- and 16-byte stores, so d_X must be
    16-byte aligned; the histogram counts fit g <= 512 only."""
    from paper_1810_13132_gb300 import Config, Mlp, Vbdr, VbdrError
    from paper_1810_13132_gb300.vbdr import _stream_ptr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    v = Vbdr(Config(k=3, num_bdr=1 << 16, log2_g=8))
    v.scan(torch.zeros((1024, 2), dtype=torch.int32, device="cuda"))
    v.slide()
    aips = torch.arange(64, dtype=torch.int32, device="cuda")
    X = torch.empty((64 * 48 + 8,), dtype=torch.bfloat16, device="cuda")
    plain = torch.empty(64, dtype=torch.float32, device="cuda")
    rc = v._L.vbdr_features(v._h, aips.data_ptr(), 64, X.data_ptr() + 8, plain.data_ptr(),
                            _stream_ptr(None))
    assert rc == -1  # 8-byte aligned rows are refused
    rc = v._L.vbdr_features(v._h, aips.data_ptr(), 64, X.data_ptr(), plain.data_ptr(),
                            _stream_ptr(None))
    assert rc == 0
    big = Vbdr(Config(k=3, num_bdr=1 << 16, log2_g=11))
    big.scan(torch.zeros((1024, 2), dtype=torch.int32, device="cuda"))
    big.slide()
    with pytest.raises(VbdrError) as e:
        big.features(aips)
    assert e.value.code == -4
    with pytest.raises(VbdrError) as e:
        big.estimate_learned(Mlp(seed=2), aips)
    assert e.value.code == -4
    torch.cuda.synchronize()
