"""dss_pairs_noalloc against the regular neighbour search.

dss_pairs_noalloc serves callers that may not allocate device memory (for
example a solver embedded in a host framework that owns every GPU
allocation): it finds the neighbour pairs using only a fixed array compiled
into the library.  Here it is called through the C ABI and its pair set is
compared, bit for bit, with the one the regular entry points
(dss_neighbour_build + dss_get_pairs) produce, on two calls in a row with
different systems, so that the later calls also show the shared array is
cleared between calls, including the cutoff mode with a range fixed in a0 and
the wider listing ranges of the electro-chemical forces.  The file name makes
pytest collect it last.
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
        (synth.small(3000, 0.52, 31), 0.8, 1e-3, 4321, {}),
        (synth.small(1200, 0.45, 32), 1.7, 1e-2, 77, {}),
        # lubrication range a fixed multiple of a0 (cutoff mode 1)
        (synth.small(2000, 0.50, 33), 1.1, 1e-3, 919, dict(lub_cutoff_mode=1, delta_lub=0.1)),
        # the electro-chemical ranges of Eq. 6-7 (20 lambda_D, 4 a0) widen the list
        (synth.small(1500, 0.48, 34), 0.6, 1e-3, 12, dict(f_er=1.0, lambda_d=0.05,
                                                         hamaker=1e-4, vdw_eps=0.01)),
    ]
    for g, gdot, dt, nstep, extra in cases:
        box = g["box"]
        p = dss.default_params(box, shear_rate=gdot, dt=dt, mu=0.5, **extra)
        n = g["a"].shape[0]
        s = dss.Suspension(g["x"], g["a"], box, p, ids=g["ids"], nstep=nstep,
                           alpha_lin=np.zeros((3, n)), alpha_ang=np.zeros((3, n)))
        s.neighbour_build()
        want = s.pairs()
        s.close()
        cap = len(want) + 64            # room for every pair (the electro-chemical ranges list many)
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
