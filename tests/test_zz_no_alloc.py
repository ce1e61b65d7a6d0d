"""qd_cdf_noalloc: prefix sums for callers that may not allocate device memory.

The entry point writes to a caller-provided device buffer and keeps its
scratch in a fixed array inside the library, so a caller whose allocator owns
the device heap (or whose loop may not allocate) can still get the FP64
prefix sums.  Its results must match qd_cdf, the allocating entry point, on
two calls in a row (the second on a different state, so stale scratch from the
first call would show).  This file is collected last on purpose.
"""
import numpy as np
import pytest

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
def test_noalloc_cdf_matches_qd_cdf_twice(prec):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream().cuda_stream
    # first a larger state spanning many scan chunks with a ragged tail, then
    # a smaller one: the second call must not see the first call's scratch
    for dims in ([3] * 11 + [5], [3, 4, 2, 5, 7]):
        psi = _state(rng, dims, prec)
        N = psi.size
        with L.Register(dims, None, prec, stream=stream) as r:
            L.qd_set_amplitudes(r.h, psi)
            want = L.qd_cdf(r.h)
            out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
            L.qd_cdf_noalloc(L.qd_info(r.h)["state"], N, prec, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= 1e-12
        assert got[-1] == pytest.approx(float(np.sum(np.abs(psi.astype(np.complex128)) ** 2)), abs=1e-12)


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
