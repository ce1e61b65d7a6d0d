"""qd_cdf_noalloc: prefix sums for callers that may not allocate device memory.

The entry point writes to a caller-provided device buffer and keeps its
scratch in a fixed array inside the library, so a caller whose allocator owns
the device heap (or whose loop may not allocate) can still get the FP64
prefix sums.  Its results must match the FP64 oracle's prefix sums and
qd_cdf, the allocating entry point, on calls in a row (each on a different
state, so stale scratch from the call before would show).  The sizes cover a
ragged last chunk, an exact multiple of the 4096-amplitude scan chunk, and
states at and just below the 2^28-amplitude limit of the fixed scratch.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def _state(rng, dims, prec):
    N = int(np.prod(dims))
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    v /= np.linalg.norm(v)
    return v.astype(np.complex64 if prec == L.QD_C64 else np.complex128)


@pytest.mark.parametrize("prec", [L.QD_C64, L.QD_C128])
def test_noalloc_cdf_matches_oracle_and_qd_cdf_in_a_row(prec):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream().cuda_stream
    # a state spanning many scan chunks with a ragged tail (885,735
    # amplitudes), an exact multiple of the chunk (4^8 = 16 x 4096), and a
    # small one: each call must not see the call before's scratch
    for dims in ([3] * 11 + [5], [4] * 8, [3, 4, 2, 5, 7]):
        psi = _state(rng, dims, prec)
        N = psi.size
        with L.Register(dims, None, prec, stream=stream) as r:
            L.qd_set_amplitudes(r.h, psi)
            want_lib = L.qd_cdf(r.h)
            out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
            L.qd_cdf_noalloc(L.qd_info(r.h)["state"], N, prec, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
        want = qo.cdf(psi.astype(np.complex128))
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= 1e-12
        assert np.max(np.abs(got - want_lib)) <= 1e-12
        assert got[-1] == pytest.approx(float(np.sum(np.abs(psi.astype(np.complex128)) ** 2)), abs=1e-12)


@pytest.mark.parametrize("dims", [[2] * 28, [5] * 12], ids=["2^28_at_limit", "5^12_ragged"])
def test_noalloc_cdf_at_and_near_scratch_limit(dims):
    # 2^28 amplitudes fill all 65,536 chunk sums exactly; 5^12 = 244,140,625
    # uses 59,605 with a ragged last chunk.  The state lives in a torch buffer
    # the register borrows; qd_cdf (allocating) and qd_cdf_noalloc are compared
    # on the device, and the grand total against an FP64 sum of |psi|^2.
    torch = pytest.importorskip("torch")
    N = int(np.prod(dims))
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    buf = torch.empty(N, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    want_dev = torch.empty(N, dtype=torch.float64, device="cuda")
    got = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    with L.Register(dims, None, L.QD_C64, dev_buf=buf.data_ptr(), dev_buf_bytes=N * 8, stream=stream) as r:
        # the register initialises the borrowed buffer; the test state is
        # written afterwards, on the same stream
        torch.cuda.synchronize()
        buf.copy_(torch.randn(N, dtype=torch.complex64, device="cuda", generator=g))
        buf /= torch.linalg.vector_norm(buf.to(torch.complex128)).to(torch.float32)
        L.qd_cdf(r.h, where=L.QD_DEVICE, dev_ptr=want_dev.data_ptr())
        for _ in range(2):  # twice in a row on the same shared scratch
            got.fill_(float("nan"))
            L.qd_cdf_noalloc(buf.data_ptr(), N, L.QD_C64, got.data_ptr(), stream)
            torch.cuda.synchronize()
            assert bool(torch.isfinite(got).all())
            assert float((got - want_dev).abs().max()) <= 1e-12
    total = float((buf.real.double() ** 2 + buf.imag.double() ** 2).sum())
    assert float(got[-1]) == pytest.approx(total, abs=1e-9)
    del buf, got, want_dev
    torch.cuda.empty_cache()


def test_noalloc_cdf_rejects_oversized_state():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(L.QuditError) as e:
        L.qd_cdf_noalloc(buf.data_ptr(), (1 << 28) + 1, L.QD_C64, out.data_ptr(), 0)
    assert e.value.code == -2
    with pytest.raises(L.QuditError) as e:
        L.qd_cdf_noalloc(buf.data_ptr(), 0, L.QD_C64, out.data_ptr(), 0)
    assert e.value.code == -2
