"""dss_pairs_noalloc against the regular neighbour search.

dss_pairs_noalloc serves callers that may not allocate device memory (for
example a solver embedded in a host framework that owns every GPU
allocation): it finds the neighbour pairs using only a fixed array compiled
into the library.  Here it is called through the C ABI and its pair set is
compared, bit for bit, with the one the regular entry points
(dss_neighbour_build + dss_get_pairs) produce, on two calls in a row with
different systems, so that the second call also shows the shared array is
cleared between calls.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sorted_pairs(v):
    v = np.asarray(v, dtype=np.int64).reshape(-1, 2)
    return v[np.lexsort((v[:, 1], v[:, 0]))]


def _noalloc(nat, x, a, ids, box, params, a_max, nstep, cap):
    import torch
    xd = torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    ad = torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    idd = torch.as_tensor(np.ascontiguousarray(ids), dtype=torch.int32, device="cuda")
    out = torch.full((cap, 2), -1, dtype=torch.int64, device="cuda")
    cnt = ctypes.c_int64(-1)
    boxc = (ctypes.c_double * 3)(*[float(b) for b in box])
    stream = torch.cuda.current_stream()
    rc = nat.load().dss_pairs_noalloc(
        ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(idd.data_ptr()),
        a.shape[0], boxc, ctypes.byref(params), float(a_max), int(nstep),
        ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(cnt), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, cnt.value, out.cpu().numpy()


def test_noalloc_pairs_equal_regular_pairs_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import _native as nat, synth
    dss.build()
    cases = [
        (synth.small(3000, 0.52, 31), 0.8, 1e-3, 4321),
        (synth.small(1200, 0.45, 32), 1.7, 1e-2, 77),
    ]
    for g, gdot, dt, nstep in cases:
        box = g["box"]
        p = dss.default_params(box, shear_rate=gdot, dt=dt, mu=0.5)
        n = g["a"].shape[0]
        s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], nstep=nstep,
                           alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
        s.neighbour_build()
        want = s.pairs()
        s.close()
        cap = 8 * n
        rc, count, out = _noalloc(nat, g["x"], g["a"], g["ids"], box, p, g["a"].max(), nstep, cap)
        assert rc == 0, nat.ERRORS.get(rc, rc)
        assert count == len(want)
        np.testing.assert_array_equal(_sorted_pairs(out[:count]), want)
        assert (out[count:] == -1).all()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import _native as nat
    dss.build()
    n = 2_100_000                       # more particles than the array has words
    box = np.array([400.0, 400.0, 400.0])
    p = dss.default_params(box)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((3, n), dtype=torch.float64, device="cuda", generator=g) * 399.0
    a = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.empty((16, 2), dtype=torch.int64, device="cuda")
    boxc = (ctypes.c_double * 3)(*box.tolist())
    cnt = ctypes.c_int64(-1)
    rc = nat.load().dss_pairs_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                      None, n, boxc, ctypes.byref(p), 1.0, 0,
                                      ctypes.c_void_p(out.data_ptr()), 16, ctypes.byref(cnt), None)
    assert rc == -10
    assert cnt.value == -1
    assert b"scratch" in nat.load().dss_strerror(rc)
