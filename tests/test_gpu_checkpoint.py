"""Checkpoint / resume: a handle restored from vbdr_save continues exactly as
the uninterrupted one (state and estimates bit for bit), mid-slice included;
a checkpoint of another configuration or a short buffer is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_resume_equals_uninterrupted(layout):
    from paper_1810_13132_gb300 import Config, Vbdr
    cfg = Config(k=7, num_bdr=(1 << 17) + 1, log2_g=7, layout=layout)
    gen = traffic.ZipfTraffic(3000, 1.1, 5000, 7, seed=91)
    slices = [_dev(gen.next_slice(150_001)) for _ in range(10)]
    aips = _dev(gen.aips)
    a = Vbdr(cfg)
    for s in slices[:5]:
        a.scan(s)
        a.slide()
    a.scan(slices[5][:40_000])  # mid-slice: part of the next slice scanned
    blob = a.save()
    b = Vbdr(cfg)
    b.load(blob)
    for v in (a, b):
        v.scan(slices[5][40_000:])
        v.slide()
    np.testing.assert_array_equal(a.estimate(aips).cpu().numpy(), b.estimate(aips).cpu().numpy())
    for s in slices[6:]:
        for v in (a, b):
            v.scan(s)
            v.slide()
        sa, sb = a.state(), b.state()
        for key in ("dr", "bs", "reg"):
            np.testing.assert_array_equal(sa[key], sb[key])
        assert a.pool_sums() == b.pool_sums()
    assert torch.equal(a.estimate(aips), b.estimate(aips))


def test_load_refuses_other_configuration_and_short_buffer():
    from paper_1810_13132_gb300 import Config, Vbdr, VbdrError
    a = Vbdr(Config(k=7, num_bdr=1 << 16, log2_g=7))
    blob = a.save()
    for other in (Config(k=8, num_bdr=1 << 16, log2_g=7), Config(k=7, num_bdr=1 << 16, log2_g=6),
                  Config(k=7, num_bdr=1 << 16, log2_g=7, layout="gsmall"),
                  Config(k=7, num_bdr=1 << 16, log2_g=7, seed=5)):
        with pytest.raises(VbdrError) as e:
            Vbdr(other).load(blob)
        assert e.value.code == -1
    with pytest.raises(VbdrError):
        Vbdr(Config(k=7, num_bdr=1 << 16, log2_g=7)).load(blob[:-1])
    with pytest.raises(VbdrError):  # a fresh handle: estimate before any slide
        Vbdr(Config(k=7, num_bdr=1 << 16, log2_g=7)).estimate(_dev(np.arange(3, dtype=np.uint32)))
