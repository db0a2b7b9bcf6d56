"""dss_step_io (upload, steps, download and stress in one call, one
synchronisation) against the separate calls it fuses: dss_load_state,
dss_step, dss_get_state, dss_stress.  The results must be bitwise equal, with
host (pinned and pageable) and device buffers, in and out the same buffers,
and with step counts that end on either buffer parity."""
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
    return dict(dss=dss, synth=synth, torch=torch)


def _pair(env, precision):
    g = env["synth"].small(3000, 0.52, 11)
    dss = env["dss"]
    p = dss.default_params(g["box"], precision=precision, mu=0.5, shear_rate=1.5, dt=1e-3)
    a = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"])
    b = dss.Suspension(g["x"], g["a"], g["box"], p, ids=g["ids"])
    a.step(5)
    b.step(5)
    return a, b, g["a"].shape[0]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["pinned", "pageable", "device"])
def test_step_io_equals_separate_calls(env, precision, kind):
    torch = env["torch"]
    a, b, n = _pair(env, precision)

    def buf():
        if kind == "pinned":
            return torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        if kind == "device":
            return torch.empty((3, n), dtype=torch.float64, device="cuda")
        return np.empty((3, n))

    sa = [buf() for _ in range(5)]
    sb = [buf() for _ in range(5)]
    ta = [torch.empty((3, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    a.get_state_into(*ta)
    b.get_state_into(*ta)
    for k in range(5):
        if kind == "device":
            sa[k].copy_(ta[k])
            sb[k].copy_(ta[k])
        else:
            v = ta[k].cpu()
            sa[k][...] = v if kind == "pinned" else v.numpy()
            sb[k][...] = v if kind == "pinned" else v.numpy()
    for nsteps in (1, 3, 2):
        # a: the fused call, in and out the same buffers
        sig_a = np.empty(9)
        a.step_io(sa, nsteps, sa, sig_a)
        # b: the separate calls
        b.load_state(*sb)
        b.step(nsteps)
        outs = [torch.empty((3, n), dtype=torch.float64, device="cuda") for _ in range(5)]
        b.get_state_into(*outs)
        sig_b = np.asarray(b.stress()).reshape(9)
        for k in range(5):
            got = sa[k].cpu().numpy() if kind != "pageable" else sa[k]
            want = outs[k].cpu().numpy()
            assert np.array_equal(got, want), (nsteps, k)
            if kind == "device":
                sb[k].copy_(outs[k])
            else:
                sb[k][...] = outs[k].cpu() if kind == "pinned" else want
        assert np.array_equal(sig_a, sig_b), nsteps
        assert a.counters()["steps_done"] == b.counters()["steps_done"]
    a.close()
    b.close()


def test_step_io_without_outputs(env):
    """out NULL: only the stress comes back; the state stays on the device."""
    torch = env["torch"]
    a, b, n = _pair(env, "mixed")
    st = [torch.empty((3, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    a.get_state_into(*st)
    sig = np.empty(9)
    a.step_io(st, 2, None, sig)
    b.step(2)
    assert np.array_equal(sig, np.asarray(b.stress()).reshape(9))
    x_a = torch.empty((3, n), dtype=torch.float64, device="cuda")
    x_b = torch.empty_like(x_a)
    a.get_state_into(x_a, *[torch.empty_like(x_a) for _ in range(4)])
    b.get_state_into(x_b, *[torch.empty_like(x_b) for _ in range(4)])
    assert torch.equal(x_a, x_b)
    a.close()
    b.close()
