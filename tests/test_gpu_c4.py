"""The 256-instance flow-curve batch (2.7 M particles; per instance N, volume
fraction and shear rate drawn as the benchmark draws them), in the launch
configuration the benchmark times (mixed precision, one handle).  For the
instances at the extremes of the sweep (largest and smallest N, densest and
loosest, fastest and slowest shear) the oracle, run on that instance alone
with its own box, Lees-Edwards offset and dashpot, checks sampled particles
one by one on inputs made without the CUDA path (seeded packing, seeded
velocities, a seeded stretch on the contacts the oracle finds): complete
neighbour sets bit-exact, forces and torques within 1e-5.  Every instance's
forces, torques and bulk stress are also checked against the oracle's full
evaluation of that instance (its cell-list search)."""
import numpy as np
import pytest

from fullsize_cases import contact_history, partners, sample, velocities
from parity import KAPPA_MIXED, MIXED_TOL, check_forces, check_stress

pytestmark = pytest.mark.gpu

NSTEP = 3_141_593


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
    bs = synth.BATCH_SPECS["c4"]
    b = synth.generate_batch(bs)
    off = np.concatenate([[0], np.cumsum(b["n"])])
    picks = sorted({int(np.argmax(b["n"])), int(np.argmin(b["n"])), int(np.argmax(b["phi"])),
                    int(np.argmin(b["phi"])), int(np.argmax(b["shear_rates"])),
                    int(np.argmin(b["shear_rates"]))})
    N = int(off[-1])
    u = np.zeros((3, N))
    w = np.zeros((3, N))
    for k in range(len(b["n"])):
        sl = slice(off[k], off[k + 1])
        u[:, sl], w[:, sl] = velocities(b["x"][:, sl], b["a"][sl], b["shear_rates"][k], seed=400 + k)
    inst = []
    keys_all, xi_all = [], []
    for k in picks:
        sl = slice(off[k], off[k + 1])
        x, a = np.ascontiguousarray(b["x"][:, sl]), b["a"][sl]
        ids = np.arange(b["n"][k], dtype=np.int32)
        po = oracle.make_params(b["boxes"][k], mu=bs.mu, kn=bs.kn, dt=bs.dt, shear_rate=b["shear_rates"][k])
        o_off = oracle.le_offset(po, NSTEP)
        idx = sample(a, m=24, seed=k)
        keys, xi = contact_history(oracle, po, o_off, x, a, ids, u[:, sl], w[:, sl], idx, seed=k)
        o = oracle.System(po, x, a, ids=ids, u=u[:, sl], w=w[:, sl], nstep=NSTEP)
        o.set_history(keys, xi)
        Fo, To, Fa, Ta = o.forces_sampled(idx, scale=True)
        want = [oracle.neighbours_of(x, a, ids, po, o_off, int(q)) + off[k] for q in idx]
        lo, hi = keys >> 32, keys & 0xffffffff
        keys_all.append(((lo + off[k]) << 32) | (hi + off[k]))
        xi_all.append(xi)
        inst.append(dict(k=k, idx=idx + off[k], Fo=Fo, To=To, Fa=Fa, Ta=Ta, want=want))
    return dict(oracle=oracle, dss=dss, b=b, bs=bs, u=u, w=w, inst=inst, off=off,
                keys=np.concatenate(keys_all), xi=np.concatenate(xi_all), keys_by_inst=dict(
                    zip(picks, keys_all)), xi_by_inst=dict(zip(picks, xi_all)))


def test_c4_sampled_instances_vs_oracle(env):
    b, bs, dss = env["b"], env["bs"], env["dss"]
    N = int(b["n"].sum())
    p = dss.default_params(precision="mixed", mu=bs.mu, kn=bs.kn, dt=bs.dt)
    s = dss.Batch(b["x"], b["a"], b["n"], b["boxes"], b["shear_rates"], p, ids=b["ids"], u=env["u"],
                  w=env["w"], nstep=NSTEP, alpha_lin=np.zeros((3, N)), alpha_ang=np.zeros((3, N)))
    s.neighbour_build()
    pairs = s.pairs()
    for c in env["inst"]:
        for q, want in zip(c["idx"], c["want"]):
            np.testing.assert_array_equal(partners(pairs, int(q)), want)
    assert len(env["keys"]) > 50
    s.set_history(env["keys"], env["xi"])
    F, T = s.forces()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    for c in env["inst"]:
        check_forces(F[:, c["idx"]], c["Fo"], c["Fa"], MIXED_TOL, KAPPA_MIXED, "force %d" % c["k"])
        check_forces(T[:, c["idx"]], c["To"], c["Ta"], MIXED_TOL, KAPPA_MIXED, "torque %d" % c["k"])
    s.close()


def test_c4_every_instance_stress_vs_oracle(env):
    """All 256 instances: every particle's force and torque and the bulk
    stress of each instance (Eq. 8) against the oracle run on that instance
    alone (its own box, offset, shear rate and dashpot; the seeded history on
    the instances that carry one)."""
    b, bs, dss, oracle = env["b"], env["bs"], env["dss"], env["oracle"]
    off = env["off"]
    N = int(b["n"].sum())
    p = dss.default_params(precision="mixed", mu=bs.mu, kn=bs.kn, dt=bs.dt)
    s = dss.Batch(b["x"], b["a"], b["n"], b["boxes"], b["shear_rates"], p, ids=b["ids"], u=env["u"],
                  w=env["w"], nstep=NSTEP, alpha_lin=np.zeros((3, N)), alpha_ang=np.zeros((3, N)))
    s.set_history(env["keys"], env["xi"])
    F, T = s.forces()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    sig, _, _ = s.batch_stress()
    s.close()
    for k in range(len(b["n"])):
        sl = slice(off[k], off[k + 1])
        x, a = np.ascontiguousarray(b["x"][:, sl]), b["a"][sl]
        ids = np.arange(b["n"][k], dtype=np.int32)
        po = oracle.make_params(b["boxes"][k], mu=bs.mu, kn=bs.kn, dt=bs.dt, shear_rate=b["shear_rates"][k])
        o = oracle.System(po, x, a, ids=ids, u=env["u"][:, sl], w=env["w"][:, sl], nstep=NSTEP, cells=True)
        if k in env["keys_by_inst"]:
            lo, hi = env["keys_by_inst"][k] >> 32, env["keys_by_inst"][k] & 0xffffffff
            o.set_history(((lo - off[k]) << 32) | (hi - off[k]), env["xi_by_inst"][k])
        Fo, To, So = o.forces()
        Fa, Ta = o.force_scale()
        check_forces(F[:, sl], Fo, Fa, MIXED_TOL, KAPPA_MIXED, "force %d" % k)
        check_forces(T[:, sl], To, Ta, MIXED_TOL, KAPPA_MIXED, "torque %d" % k)
        check_stress(sig[k], So, MIXED_TOL, what="stress %d" % k)
