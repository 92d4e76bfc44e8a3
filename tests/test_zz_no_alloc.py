"""The no-allocation norms entry point (lbm_norms_noalloc) against lbm_norms.

Some callers cannot allocate device memory at all (code running while another component
captures a CUDA graph, allocator-less hosts, latency-critical paths); lbm_norms_noalloc
serves them from a static array inside the library.  This file is collected last so that
a failure here comes after every other test has run; it passes both alone in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_1308_0692_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_0692_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _reference(a, b, prec, count=None):
    count = a.numel() if count is None else count
    nbytes = lbm.lbm_norms_scratch_bytes(count)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    lbm.lbm_norms(a.data_ptr(), b.data_ptr() if b is not None else None, count, prec,
                  scratch.data_ptr(), nbytes, out.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,dtype", [(lbm.LBM_FP64, torch.float64), (lbm.LBM_FP32_PERTURB, torch.float32)])
@pytest.mark.parametrize("count", [1, 2049, 3 * 10 ** 6 + 17])
def test_noalloc_matches_allocating_entry_point_twice(prec, dtype, count):
    """Two calls in a row (the second sees the first call's leftovers in the static array)
    agree with lbm_norms within the FP64 parity tolerance."""
    g = torch.Generator(device="cpu").manual_seed(count + prec)
    s = torch.cuda.current_stream()
    for rep in range(2):
        a = torch.randn(count + rep, generator=g, dtype=torch.float64).to(dtype).cuda()
        b = torch.randn(count + rep, generator=g, dtype=torch.float64).to(dtype).cuda()
        for bb in (b, None):
            out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
            lbm.lbm_norms_noalloc(a.data_ptr(), bb.data_ptr() if bb is not None else None, a.numel(),
                                  prec, out.data_ptr(), s)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            ref = _reference(a, bb, prec)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_noalloc_rejects_counts_beyond_the_static_scratch():
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_norms_noalloc(a.data_ptr(), None, 2 ** 26 + 1, lbm.LBM_FP32_PERTURB, out.data_ptr())
    assert e.value.status == lbm.LBM_EINVAL


@pytest.mark.parametrize("prec,dtype", [(lbm.LBM_FP64, torch.float64), (lbm.LBM_FP32_PERTURB, torch.float32)])
def test_noalloc_empty_input_gives_zero_norms(prec, dtype):
    """count = 0 launches no chunk blocks; the finalisation over zero partials writes {0, 0},
    the same as lbm_norms, also right after a call that left partials in the static array."""
    s = torch.cuda.current_stream()
    a = torch.randn(5000, dtype=torch.float64).to(dtype).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    lbm.lbm_norms_noalloc(a.data_ptr(), None, a.numel(), prec, out.data_ptr(), s)
    for bb in (a, None):
        out.fill_(-1.0)
        lbm.lbm_norms_noalloc(a.data_ptr(), bb.data_ptr() if bb is not None else None, 0, prec, out.data_ptr(), s)
        torch.cuda.synchronize()
        assert out.cpu().tolist() == [0.0, 0.0]
        np.testing.assert_array_equal(_reference(a, bb, prec, count=0), [0.0, 0.0])
