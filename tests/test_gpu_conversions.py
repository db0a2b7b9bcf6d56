"""The sort kernels' conversions by integer operations (f32_rn, the
double-float split, float -> double, int -> double, the cell-coordinate
floor) against CUDA's own conversions, bit for bit, over random doubles of
every magnitude, exact rounding ties (both parities), the float range's ends,
signed zeros, infinities, and products within ulps of an integer."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import _native
    dss.build()
    return dict(torch=torch, lib=_native.load())


def _inputs(inv):
    rng = np.random.default_rng(17)
    parts = []
    # every magnitude, both signs
    e = rng.uniform(-140, 140, size=200000)
    parts.append(np.sign(rng.uniform(-1, 1, size=e.size)) * np.exp2(e) * rng.uniform(1, 2, size=e.size))
    # exact ties: the 29 discarded bits 1000...0, the kept bits even and odd
    b = rng.integers(0, 1 << 52, size=20000, dtype=np.uint64)
    b = (b & ~np.uint64((1 << 29) - 1)) | np.uint64(1 << 28)
    ex = rng.integers(897, 1151, size=b.size).astype(np.uint64)
    parts.append(((ex << np.uint64(52)) | b).view(np.float64))
    # ties and near-ties next to a carry into the exponent
    b2 = np.full(1000, (1 << 52) - 1, dtype=np.uint64) - rng.integers(0, 1 << 30, size=1000).astype(np.uint64)
    parts.append(((ex[:1000] << np.uint64(52)) | b2).view(np.float64))
    # the ends of the float range, zeros, infinities
    fmax = float(np.finfo(np.float32).max)
    fmin = float(np.finfo(np.float32).tiny)
    ends = [0.0, -0.0, np.inf, -np.inf, fmax, -fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -23),
            fmin, -fmin, fmin * 0.5, fmin * (1 - 2.0 ** -30), 2.0 ** -75, 2.0 ** -74, 1e-300, 1e300]
    parts.append(np.array(ends))
    # cell-local positions and products within a few ulps of an integer
    k = rng.integers(0, 1023, size=50000).astype(np.float64)
    cs = 1.0 / inv
    near = k * cs
    parts.append(near)
    parts.append(np.nextafter(near, np.inf))
    parts.append(np.nextafter(near, -np.inf))
    parts.append(near * (1 + rng.uniform(-4e-7, 4e-7, size=k.size)))
    parts.append(rng.uniform(0, 1023 * cs, size=50000))
    return np.concatenate(parts)


def test_conversions_match_hardware(env):
    torch, lib = env["torch"], env["lib"]
    inv = 1.0 / 2.0515
    v = torch.from_numpy(_inputs(inv)).cuda()
    n = v.numel()
    hi = torch.empty(n, dtype=torch.float32, device="cuda")
    shi, slo = torch.empty_like(hi), torch.empty_like(hi)
    back = torch.empty(n, dtype=torch.float64, device="cuda")
    fl = torch.empty(n, dtype=torch.int32, device="cuda")
    ints = torch.from_numpy(np.concatenate([np.arange(0, 70000), np.random.default_rng(3).integers(
        0, 2 ** 31 - 1, size=n - 70000)]).astype(np.int32)).cuda()
    ints_out = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = lib.dss_selftest_conversions(v.data_ptr(), n, inv, hi.data_ptr(), shi.data_ptr(), slo.data_ptr(),
                                      back.data_ptr(), fl.data_ptr(), ints.data_ptr(), ints_out.data_ptr(),
                                      None)
    assert rc == 0
    want_hi = v.to(torch.float32)
    want_lo = (v - want_hi.to(torch.float64)).to(torch.float32)
    bits = lambda t: t.view(torch.int32) if t.dtype == torch.float32 else t.view(torch.int64)
    assert torch.equal(bits(hi), bits(want_hi))
    assert torch.equal(bits(shi), bits(want_hi))
    finite = torch.isfinite(v)
    assert torch.equal(bits(slo[finite]), bits(want_lo[finite]))
    assert torch.equal(bits(back), bits(want_hi.to(torch.float64)))
    assert torch.equal(bits(ints_out), bits(ints.to(torch.float64)))
    # the cell coordinate where the FP64 floor is an int
    p = v * inv
    ok = finite & (p.abs() < 2.0 ** 30)
    assert torch.equal(fl[ok], torch.floor(p[ok]).to(torch.int32))
    # the near-integer products took both paths
    assert int(ok.sum()) > 250000
