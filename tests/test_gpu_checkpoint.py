"""Checkpoint / resume and the cell-size autotuner.

The sorted order inside the library depends only on positions and ids, so a
run resumed from a checkpoint must repeat the uninterrupted run bit for bit
(state, contact history and stress), and the autotuner, which runs its trial
steps from a checkpoint, must leave the state exactly as it found it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2108_01013_gb300 as dss
    from paper_2108_01013_gb300 import synth
    dss.build()
    synth.build()
    return dict(dss=dss, synth=synth)


def _state(s):
    return {k: v.cpu().numpy() for k, v in s.state().items()}


def _same(s1, s2):
    a, b = _state(s1), _state(s2)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    k1, x1 = s1.history()
    k2, x2 = s2.history()
    assert np.array_equal(k1, k2) and np.array_equal(x1, x2)
    assert np.array_equal(s1.stress(), s2.stress())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_is_bit_exact(env, precision):
    g = env["synth"].small(1500, 0.54, 41)
    box = g["box"]
    p = env["dss"].default_params(box, mu=1.0, shear_rate=5.0, precision=precision)
    a = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    a.step(20)
    ck = a.save()
    a.step(25)
    b = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    b.step(3)                       # a different state, overwritten by the checkpoint
    b.load(ck)
    assert b.counters()["nstep"] == 20
    b.step(25)
    assert a.counters()["ncontacts"] > 10
    _same(a, b)
    a.close()
    b.close()


def test_checkpoint_rejects_other_configurations(env):
    dss = env["dss"]
    g = env["synth"].small(800, 0.5, 42)
    box = g["box"]
    s = dss.Suspension(g["x"], g["a"], box, dss.default_params(box, mu=0.5))
    ck = s.save()
    t = dss.Suspension(g["x"], g["a"], box, dss.default_params(box, mu=0.6))
    with pytest.raises(dss.DssError) as e:
        t.load(ck)
    assert e.value.code == -1
    bad = bytearray(ck)
    bad[0] ^= 0xFF
    with pytest.raises(dss.DssError) as e:
        s.load(bytes(bad))
    assert e.value.code == -1
    with pytest.raises(dss.DssError) as e:
        s.load(ck[:len(ck) - 8])
    assert e.value.code == -1
    s.close()
    t.close()


def test_batch_resume_keeps_mean_stress(env):
    dss = env["dss"]
    gs = [env["synth"].small(n, phi, seed) for n, phi, seed in [(600, 0.5, 43), (900, 0.45, 44)]]
    x = np.concatenate([g["x"] for g in gs], axis=1)
    a = np.concatenate([g["a"] for g in gs])
    args = (x, a, [600, 900], [g["box"] for g in gs], [0.5, 8.0], dss.default_params(precision="mixed"))
    b1 = dss.Batch(*args)
    b1.step(10)
    ck = b1.save()
    b1.step(10)
    b2 = dss.Batch(*args)
    b2.load(ck)
    b2.step(10)
    s1, m1, n1 = b1.batch_stress()
    s2, m2, n2 = b2.batch_stress()
    assert n1 == n2 == 20
    assert np.array_equal(s1, s2) and np.array_equal(m1, m2)
    _same(b1, b2)


def test_autotune_restores_state_and_picks_a_candidate(env):
    g = env["synth"].small(3000, 0.52, 45)
    box = g["box"]
    p = env["dss"].default_params(box, mu=0.5, precision="mixed")
    s = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    s.step(5)
    before = _state(s)
    hk, hx = s.history()
    cs, trials = s.autotune(trial_steps=5, factors=[1.0, 1.2, 1.45])
    assert len(trials) == 3 and all(np.isfinite(v) and v > 0 for v in trials.values())
    best = min(trials, key=trials.get)
    assert cs == pytest.approx(best * (2 * g["a"].max() + 0.05 * g["a"].max()), rel=1e-6)
    after = _state(s)
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    k2, x2 = s.history()
    assert np.array_equal(hk, k2) and np.array_equal(hx, x2)
    assert s.counters()["nstep"] == 5
    s.step(5)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_step_graphs_repeat_single_steps(env, precision):
    """dss_step(n) sends runs of 8 steps as one graph launch; the trajectory,
    history and stress equal n single-step calls bit for bit (the same
    kernels in the same order), including a remainder of single steps."""
    g = env["synth"].small(2500, 0.53, 47)
    box = g["box"]
    p = env["dss"].default_params(box, mu=0.7, shear_rate=3.0, precision=precision)
    a = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    b = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    a.step(21)
    for _ in range(21):
        b.step(1)
    _same(a, b)
    assert a.counters()["steps_done"] == b.counters()["steps_done"] == 21
    a.close()
    b.close()


def test_kernel_shape_autotune_keeps_the_trajectory(env):
    """dss_autotune_kernels times the four kernel shapes (pair-kernel blocks
    per SM 3 or 4, enumeration candidate loop plain or screened), keeps the fastest
    and restores the state; the shapes change neither the pairs nor the
    arithmetic, so the run continues bit for bit as an untuned one."""
    g = env["synth"].small(3000, 0.52, 48)
    box = g["box"]
    p = env["dss"].default_params(box, mu=0.5, precision="mixed")
    a = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    b = env["dss"].Suspension(g["x"], g["a"], box, p, ids=g["ids"])
    a.step(5)
    b.step(5)
    choice, trials = a.autotune_kernels(trial_steps=5)
    assert choice in trials and len(trials) == 4
    assert all(np.isfinite(v) and v > 0 for v in trials.values())
    assert trials[choice] == min(trials.values())
    _same(a, b)
    a.step(10)
    b.step(10)
    _same(a, b)
    a.close()
    b.close()
