"""Failure detection and recovery, without faulting the GPU.

- A device wait whose predecessor never publishes gives up after its time
  limit and reports DSS_ERR_TIMEOUT; the context stays usable.
- Non-finite input (a NaN injected on the host) is reported as
  DSS_ERR_NONFINITE and the failed step is not committed.
- A pair-capacity overflow inside dss_step is recovered by growing the pair
  buffers, with the same trajectory as a run that never overflowed.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import _native as nat, synth
    dss.build()
    synth.build()
    return dict(dss=dss, nat=nat, synth=synth, torch=torch)


def test_bounded_wait_reports_timeout_and_context_survives(env):
    lib = env["nat"].load()
    t0 = time.perf_counter()
    rc = lib.dss_selftest_bounded_wait(None)
    dt = time.perf_counter() - t0
    assert rc == -7, env["nat"].ERRORS.get(rc, rc)
    assert 0.3 < dt < 10.0
    # the device still works: a normal handle steps
    g = env["synth"].small(600, 0.5, 71)
    s = env["dss"].Suspension(g["x"], g["a"], g["box"], env["dss"].default_params(g["box"]))
    s.step(3)
    assert s.counters()["steps_done"] == 3
    s.close()


def test_nan_injection_is_reported_and_not_committed(env):
    dss = env["dss"]
    g = env["synth"].small(800, 0.5, 72)
    box = g["box"]
    n = g["a"].shape[0]
    s = dss.Suspension(g["x"], g["a"], box, dss.default_params(box))
    s.step(4)
    before = {k: v.cpu().numpy() for k, v in s.state().items()}
    u = before["u"].copy()
    u[0, 17] = np.nan
    s.load_state(before["x"], u, before["w"], before["al"], before["aw"])
    with pytest.raises(dss.DssError) as e:
        s.step(2)
    assert e.value.code == -4
    c = s.counters()
    assert c["steps_done"] == 4 and c["nstep"] == 4
    after = s.state()["x"].cpu().numpy()
    assert np.array_equal(after, before["x"])
    # a clean state steps again
    s.load_state(before["x"], before["u"], before["w"], before["al"], before["aw"])
    s.step(2)
    assert s.counters()["steps_done"] == 6
    # set_state with a non-finite velocity fails at its force evaluation
    u0 = np.zeros((3, n))
    u0[1, 3] = np.inf
    with pytest.raises(dss.DssError) as e:
        dss.Suspension(g["x"], g["a"], box, dss.default_params(box), u=u0)
    assert e.value.code == -4
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pair_capacity_overflow_recovers(env, precision):
    dss = env["dss"]
    g = env["synth"].small(1500, 0.55, 73)
    box = g["box"]
    p_small = dss.default_params(box, precision=precision, mu=1.0, pair_capacity=1)
    p_big = dss.default_params(box, precision=precision, mu=1.0)
    a = dss.Suspension(g["x"], g["a"], box, p_small, ids=g["ids"],
                       alpha_lin=np.zeros((3, 1500)), alpha_ang=np.zeros((3, 1500)))
    b = dss.Suspension(g["x"], g["a"], box, p_big, ids=g["ids"],
                       alpha_lin=np.zeros((3, 1500)), alpha_ang=np.zeros((3, 1500)))
    small_bytes = a.device_bytes()
    a.step(10)
    b.step(10)
    assert a.counters()["steps_done"] == 10
    assert a.device_bytes() > small_bytes          # the pair buffers grew
    sa, sb = a.state(), b.state()
    for k in sa:
        assert env["torch"].equal(sa[k], sb[k]), k
    a.close()
    b.close()
