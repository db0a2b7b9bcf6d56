"""Batched instances: K independent suspensions (each its own box, packing
fraction, particle count and shear rate, hence its own Lees-Edwards offset and
dashpot) advanced in one handle.  Every instance must match the FP64 oracle
run of that instance alone: pair sets bit for bit, FP64 forces, torques and
stresses within 1e-10, mixed precision within 1e-5 (per particle and per
stress component, tests/parity.py); and a batched run must match the
single-instance runs of its members step for step."""
import numpy as np
import pytest

from parity import (FP64_TOL, KAPPA_FP64, KAPPA_MIXED, MIXED_TOL, check_forces, check_stress)

pytestmark = pytest.mark.gpu

# n, phi, seed, shear rate
MEMBERS = [(700, 0.45, 11, 0.37), (1300, 0.55, 12, 3.1), (300, 0.50, 13, 25.0), (901, 0.40, 14, 0.02)]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import synth
    oracle.build()
    dss.build()
    synth.build()
    return dict(oracle=oracle, dss=dss, synth=synth, torch=torch)


def _members(env, members=MEMBERS):
    out = []
    for n, phi, seed, gdot in members:
        g = env["synth"].small(n, phi, seed)
        out.append(dict(g=g, gdot=gdot, n=n))
    return out


def _offsets(ms):
    return np.concatenate([[0], np.cumsum([m["n"] for m in ms])])


def _batch(env, ms, precision="fp64", nstep=0, states=None, **kw):
    off = _offsets(ms)
    if states is None:
        x = np.concatenate([m["g"]["x"] for m in ms], axis=1)
        extra = dict(alpha_lin=np.zeros((3, off[-1])), alpha_ang=np.zeros((3, off[-1])))
    else:
        x = np.concatenate([s["x"] for s in states], axis=1)
        extra = {k: np.concatenate([s[src] for s in states], axis=1)
                 for k, src in (("u", "u"), ("w", "w"), ("alpha_lin", "al"), ("alpha_ang", "aw"))}
    a = np.concatenate([m["g"]["a"] for m in ms])
    ids = np.concatenate([m["g"]["ids"] + off[k] for k, m in enumerate(ms)]).astype(np.int32)
    p = env["dss"].default_params(precision=precision, **kw)
    return env["dss"].Batch(x, a, [m["n"] for m in ms], [m["g"]["box"] for m in ms],
                            [m["gdot"] for m in ms], p, ids=ids, nstep=nstep, **extra)


def test_batch_pairs_bit_exact(env):
    ms = _members(env)
    nstep = 4321
    b = _batch(env, ms, dt=1e-3, nstep=nstep)
    b.neighbour_build()
    got = b.pairs()
    off = _offsets(ms)
    total = 0
    for k, m in enumerate(ms):
        g = m["g"]
        po = env["oracle"].make_params(g["box"], shear_rate=m["gdot"], dt=1e-3)
        lo_off = env["oracle"].le_offset(po, nstep)
        want = env["oracle"].pairs_bruteforce(g["x"], g["a"], g["ids"], po, lo_off) + off[k]
        assert len(want) > m["n"] // 3
        sel = (got[:, 0] >= off[k]) & (got[:, 0] < off[k + 1])
        assert ((got[sel] >= off[k]) & (got[sel] < off[k + 1])).all()   # no pair across instances
        np.testing.assert_array_equal(got[sel], want)
        total += len(want)
    assert total == len(got)
    b.close()


@pytest.mark.parametrize("precision,tol,kappa", [("fp64", FP64_TOL, KAPPA_FP64),
                                                 ("mixed", MIXED_TOL, KAPPA_MIXED)])
def test_batch_forces_stress_and_step_vs_oracle(env, precision, tol, kappa):
    ms = _members(env)
    off = _offsets(ms)
    orcs, states, keys, xis = [], [], [], []
    for k, m in enumerate(ms):
        g = m["g"]
        po = env["oracle"].make_params(g["box"], mu=1.0, shear_rate=m["gdot"])
        o = env["oracle"].System(po, g["x"], g["a"], ids=g["ids"])
        o.init_accel()
        o.step(25)
        kk, xx = o.get_history()
        lo, hi = kk >> 32, kk & 0xffffffff
        keys.append(((lo + off[k]) << 32) | (hi + off[k]))
        xis.append(xx)
        orcs.append(o)
        states.append(o.get_state())
    b = _batch(env, ms, precision=precision, nstep=orcs[0].nstep, states=states, mu=1.0)
    b.set_history(np.concatenate(keys), np.concatenate(xis))
    F, T = b.forces()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    sig, _, _ = b.batch_stress()
    for k, o in enumerate(orcs):
        Fo, To, So = o.forces()
        Fa, Ta = o.force_scale()
        check_forces(F[:, off[k]:off[k + 1]], Fo, Fa, tol, kappa, "force %d" % k)
        check_forces(T[:, off[k]:off[k + 1]], To, Ta, tol, kappa, "torque %d" % k)
        check_stress(sig[k], So, tol, what="stress %d" % k)
    assert sum(o.ncontacts for o in orcs) > 20
    # three steps; the mean stress of the batch is the mean of the instances' steps
    b.batch_stress(reset=True)
    sums = [np.zeros((3, 3)) for _ in orcs]
    b.step(3)
    for _ in range(3):
        for k, o in enumerate(orcs):
            o.step(1)
            sums[k] += o.get_forces()[2]
    st = b.state()
    sig, mean, steps = b.batch_stress()
    assert steps == 3
    for k, o in enumerate(orcs):
        so = o.get_state()
        box = ms[k]["g"]["box"]
        d = np.abs(st["x"].cpu().numpy()[:, off[k]:off[k + 1]] - so["x"])
        d = np.minimum(d, box[:, None] - d)
        assert d.max() < (1e-12 if precision == "fp64" else 1e-9)
        Fa, _ = o.force_scale()
        mass = 4.0 / 3.0 * np.pi * ms[k]["g"]["a"] ** 3
        check_forces(st["al"].cpu().numpy()[:, off[k]:off[k + 1]], so["al"], Fa / mass, tol, kappa,
                     "alpha %d" % k)
        check_stress(sig[k], o.get_forces()[2], tol, what="stress %d" % k)
        check_stress(mean[k], sums[k] / 3, tol, what="mean stress %d" % k)
    b.close()


def test_batch_matches_single_instance_runs(env):
    """Mixed precision, 40 steps: every member of the batch stays with its
    own single-instance run (same library, K = 1).  The two runs group the
    owners into warps differently (an instance starts anywhere in a warp of
    the batch), so their FP32 sums round differently; the positions stay
    within 1e-8 (measured ~1e-9), the mean stresses within 1e-5."""
    ms = _members(env)
    off = _offsets(ms)
    b = _batch(env, ms, precision="mixed", mu=0.5)
    b.step(40)
    xb = b.state()["x"].cpu().numpy()
    _, mb, steps = b.batch_stress()
    assert steps == 40
    for k, m in enumerate(ms):
        s = _batch(env, [m], precision="mixed", mu=0.5)
        s.step(40)
        xs = s.state()["x"].cpu().numpy()
        _, msg, _ = s.batch_stress()
        box = m["g"]["box"]
        d = np.abs(xb[:, off[k]:off[k + 1]] - xs)
        d = np.minimum(d, box[:, None] - d)
        assert d.max() < 1e-8
        check_stress(mb[k], msg[0], MIXED_TOL, what="mean stress %d" % k)
        s.close()
    b.close()


def test_batch_rejects_bad_layouts(env):
    dss = env["dss"]
    ms = _members(env, [(300, 0.45, 21, 1.0), (400, 0.45, 22, 2.0)])
    # an instance below the minimum size
    small = _members(env, [(300, 0.45, 21, 1.0), (200, 0.45, 23, 2.0)])
    with pytest.raises(dss.DssError) as e:
        _batch(env, small)
    assert e.value.code == -1
    # ids that leave their instance's range
    off = _offsets(ms)
    x = np.concatenate([m["g"]["x"] for m in ms], axis=1)
    a = np.concatenate([m["g"]["a"] for m in ms])
    ids = np.arange(off[-1], dtype=np.int32)
    ids[[0, off[1]]] = ids[[off[1], 0]]
    p = dss.default_params()
    with pytest.raises(dss.DssError) as e:
        dss.Batch(x, a, [m["n"] for m in ms], [m["g"]["box"] for m in ms], [1.0, 2.0], p, ids=ids)
    assert e.value.code == -1
    # a position inside the other instance's (larger) box but outside its own
    boxes = [m["g"]["box"] for m in ms]
    assert boxes[1][0] > boxes[0][0]
    x2 = x.copy()
    x2[0, 0] = 0.5 * (boxes[0][0] + boxes[1][0])
    with pytest.raises(dss.DssError) as e:
        dss.Batch(x2, a, [m["n"] for m in ms], boxes, [1.0, 2.0], p)
    assert e.value.code == -1


def test_adjoint_refuses_batched_handles(env):
    """The reverse sweep tapes one instance: a batch is refused (DSS_ERR_ARG)
    and left usable."""
    ms = _members(env, MEMBERS[:2])
    b = _batch(env, ms, dt=1e-3)
    with pytest.raises(RuntimeError, match="DSS_ERR_ARG"):
        b.adjoint(2, np.zeros((2, 9)))
    b.step(2)
    assert b.counters()["steps_done"] == 2
    b.close()
