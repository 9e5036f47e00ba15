"""Serving with continuous batching: every request of a mixed stream is
checked against the FP64 oracle element by element (its own kind, mode list,
nu, force and step count from the same FP32 start); its final fields are the
same, bit for bit, when it is served alone and when it shares the GPU with a
mix of others that arrive while it runs; admission waits for HBM budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00437_gb300 import build
    build.build()


def _stream(n=14, rate=400.0, seed=5):
    from paper_1803_00437_gb300 import serve
    return serve.make_requests(n, rate, seed, side_range=(64, 320), step_range=(40, 400))


def _same(a, b):
    for k in a:
        x, y = np.asarray(a[k], dtype=float), np.asarray(b[k], dtype=float)
        if not np.allclose(x, y, rtol=1e-9, atol=1e-15):
            return False
    return True


def _initial_fields(req):
    """The request's start as the device evaluates it: its transverse modes
    (rest for a channel), rounded to FP32 once."""
    from paper_1803_00437_gb300 import inputs
    from parity_util import as_f32
    if req.modes:
        return as_f32(inputs.transverse_modes(req.nx, req.ny, req.modes))
    z = np.zeros((req.ny, req.nx))
    return as_f32((z, z, z))


@pytest.fixture(scope="module")
def served_mix():
    from paper_1803_00437_gb300 import serve
    mix = serve.Server(hbm_budget=256 << 20, max_slots=16, max_side=512, run_steps=32,
                       return_fields=True)
    done = mix.serve(_stream())
    return done


def test_every_served_request_matches_the_oracle(served_mix, oracle):
    """Each request's final fields against the oracle run of its own
    configuration.  Tolerance (FP32): 1e-5 of the initial wave amplitude for
    waves; channels start at rest, so their scale is the oracle's final
    max |u|, with the FP32 forced-flow bound max(1e-5, 6e-8 n) (each step adds
    F to u with a relative rounding of ~6e-8 of u)."""
    from paper_1803_00437_gb300 import serve
    from parity_util import amplitude, max_err, oracle_run
    done = served_mix
    assert len(done) == 14 and {r.kind for r in done} == set(serve.KINDS)
    for r in done:
        f = _initial_fields(r)
        ref = oracle_run(oracle, r.config("fd5"), f, r.steps)
        got = [a.astype(np.float64) for a in r.result["fields"]]
        if r.kind == "poiseuille":
            scale = max(float(np.abs(ref[1]).max()), 1e-30)
            tol = max(1e-5, 6e-8 * r.steps)
        else:
            scale, tol = amplitude(f), 1e-5
        err = max_err(got, ref, scale)
        assert err <= tol, (r.rid, r.kind, r.nx, r.ny, r.steps, err)


def test_results_alone_equal_results_in_the_mix(served_mix):
    from paper_1803_00437_gb300 import serve
    done = served_mix
    # several requests overlapped on the device
    spans = sorted((r.admitted, r.finished) for r in done)
    assert any(a2 < f1 for (a1, f1), (a2, f2) in zip(spans, spans[1:]))
    for r in done:
        alone = serve.Server(hbm_budget=64 << 20, max_slots=1, max_side=512, run_steps=32,
                             return_fields=True)
        solo = _stream()[r.rid]
        solo.arrival = 0.0
        (res,) = alone.serve([solo])
        for a, b in zip(r.result["fields"], res.result["fields"]):
            assert np.array_equal(a, b), (r.rid, r.kind)
        scalars = {k: v for k, v in r.result.items() if k != "fields"}
        assert _same(scalars, res.result), (r.rid, r.kind, scalars, res.result)


def test_admission_waits_for_budget():
    from paper_1803_00437_gb300 import serve
    reqs = serve.make_requests(10, 1e6, 9, side_range=(200, 256), step_range=(64, 128))
    srv = serve.Server(hbm_budget=8 << 20, max_slots=8, max_side=256, run_steps=32)
    done = srv.serve(reqs)
    assert len(done) == 10
    assert max(r.admitted - r.arrival for r in done) > 0  # some waited for space
    assert all(np.isfinite(r.result["max_u"]) for r in done)


def test_poiseuille_request_approaches_parabola():
    """A channel request driven to steady state returns u_max close to the
    target 0.05 used to set its force (Sec. 3-c)."""
    from paper_1803_00437_gb300 import serve
    nu = 0.1
    req = serve.Request(0, "poiseuille", 64, 16, 3000, nu, 0.0, [],
                        (8 * nu * 0.05 / 16 ** 2, 0.0))
    srv = serve.Server(hbm_budget=16 << 20, max_slots=2, max_side=64, run_steps=64)
    (r,) = srv.serve([req])
    assert abs(r.result["max_u"] / 0.05 - 1.0) < 0.05
