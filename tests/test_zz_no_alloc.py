"""vbdr_estimate_registers_noalloc: estimates without any device allocation.

The entry point serves callers that cannot allocate device memory where they
need an estimate (all their memory is reserved up front by their own
allocator, or allocation is forbidden once their loop runs), so it works in
a fixed array compiled into the library.  This test calls it through the C ABI
on a register array built by a handle, twice in a row with different inputs,
and checks both results against the handle's own vbdr_estimate within the
estimate tolerance of the parity tests.  It lives in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

EST_RTOL = 1e-6


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _check_close(got, want):
    got = got.cpu().numpy().astype(np.float64)
    want = want.cpu().numpy().astype(np.float64)
    err = np.abs(got - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= EST_RTOL, (err.max(), int(err.argmax()))


def test_noalloc_estimate_matches_handle_estimate_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_13132_gb300 import Config, Vbdr
    from paper_1810_13132_gb300.vbdr import estimate_registers_noalloc

    torch.cuda.set_device(0)
    seed = 0x1234567
    Z, b = (1 << 18) + 5, 8
    gen = traffic.ZipfTraffic(20000, 1.05, 200000, 6, seed=404, repeat_frac=0.1)
    v = Vbdr(Config(k=6, num_bdr=Z, log2_g=b, seed=seed))
    for _ in range(4):
        v.scan(_dev(gen.next_slice(1 << 20)))
        v.slide()
    reg1 = torch.from_numpy(v.registers()).cuda()
    aips1 = _dev(gen.aips)
    want1 = v.estimate(aips1)

    out = torch.empty(aips1.numel(), dtype=torch.float32, device="cuda")
    estimate_registers_noalloc(reg1, Z, b, seed, aips1, out)
    torch.cuda.synchronize()
    _check_close(out, want1)

    # second call in a row: other registers (one more slice), other hosts
    v.scan(_dev(gen.next_slice(1 << 20)))
    v.slide()
    reg2 = torch.from_numpy(v.registers()).cuda()
    aips2 = _dev(np.ascontiguousarray(gen.aips[::-1][:7777]))
    want2 = v.estimate(aips2)
    out2 = torch.empty(aips2.numel(), dtype=torch.float32, device="cuda")
    estimate_registers_noalloc(reg2, Z, b, seed, aips2, out2)
    torch.cuda.synchronize()
    _check_close(out2, want2)
    v.close()


def test_noalloc_rejects_sizes_beyond_its_fixed_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_13132_gb300 import VbdrError
    from paper_1810_13132_gb300.vbdr import estimate_registers_noalloc
    reg = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    aips = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    with pytest.raises(VbdrError) as e:
        estimate_registers_noalloc(reg, 1 << 12, 10, 1, aips, out)  # g = 1024 > 512
    assert e.value.code == -4
