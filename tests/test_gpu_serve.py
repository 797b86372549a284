"""The request loop (bem_server_*): every request's result is the same when
it runs alone and when it is merged into a batch with other requests and
runs next to other scenes' solves, within the solved-trace bar (1e-6
relative l2), and equal to the oracle's dense solve; admission under a
device-memory budget evicts idle scenes and refuses requests that can never
fit."""
import numpy as np
import pytest

from oracle import pmchwt, rayleigh
from synth import scenes

pytestmark = pytest.mark.gpu

OMEGA_RHO0 = 2.6
TOL = 1e-10


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def api():
    from paper_1910_01011_gb300 import api, build
    build.build()
    return api


def transducer(seed):
    return scenes.bowl_transducer(seed=seed, n_elem=6, R=4.0, aperture=3.0, piston_radius=0.3, gap=0.05)


SCENES = {
    "sphere": lambda: scenes.sphere_scene(2),
    "two": lambda: scenes.two_sphere_scene(1),
    "shell": lambda: scenes.shell_scene(1),
}


def make_server(api, names, **kw):
    kw.setdefault("slots", 2)
    kw.setdefault("max_batch_rhs", 8)
    kw.setdefault("hbm_budget_bytes", 8 << 30)
    srv = api.Server(precision=1, tol=TOL, **kw)
    ids = {}
    for i, name in enumerate(names):
        s = SCENES[name]()
        ids[name] = srv.add_scene(s, transducer=transducer(i), omega_rho0=OMEGA_RHO0, r_eps=0.2)
    return srv, ids


def oracle_solution(name, seed, w):
    s = SCENES[name]()
    tr = transducer(seed)
    A = pmchwt.assemble(s)
    b = pmchwt.rhs(s, rayleigh.field(tr, w, s.k0, OMEGA_RHO0, 1.0))
    return np.linalg.solve(A, b)


def test_result_same_alone_and_in_the_mix(api):
    names = ["sphere", "two", "shell"]
    rng = np.random.default_rng(5)
    wA = np.exp(2j * np.pi * rng.random((2, 6)))
    # alone
    srv, ids = make_server(api, names)
    h = srv.submit(ids["two"], wA)
    assert srv.wait(h, 600) == 2
    U_alone, rep_alone = srv.result(h, 2, ids["two"])
    assert rep_alone["batch_exc"] == 2
    srv.close()
    # in the mix: 14 requests over three scenes, A in the middle
    srv, ids = make_server(api, names)
    plan = []
    for i in range(14):
        name = names[i % 3] if i != 7 else "two"
        w = wA if i == 7 else np.exp(2j * np.pi * rng.random((1 + i % 3, 6)))
        plan.append((name, w, srv.submit(ids[name], w)))
    out = {}
    for name, w, h in plan:
        assert srv.wait(h, 900) == 2
        out[h] = srv.result(h, w.shape[0], ids[name])
    st = srv.stats()
    srv.close()
    U_mix, rep_mix = out[plan[7][2]]
    assert rel(U_mix, U_alone) < 1e-6
    # requests were merged and scenes shared the GPU
    assert st["completed"] == 14 and st["failed"] == 0
    assert st["batches"] < 14 and st["mean_batch_exc"] > 1
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # every excitation of a few requests against the oracle's dense solve
    for k in (0, 7, 13):
        name, w, h = plan[k]
        U, _ = out[h]
        seed = names.index(name)
        for r in range(w.shape[0]):
            assert rel(U[r], oracle_solution(name, seed, w[r])) < 1e-6, (k, r)


@pytest.mark.parametrize("name,n_exc,mode,batch", [("sphere", 1, 0, 0), ("shell", 3, 0, 4), ("two", 5, 1, 8),
                                                   ("sphere", 2, 1, 0)])
def test_memory_estimate_bounds_the_peak(api, name, n_exc, mode, batch):
    """The admission estimate is an upper bound of what a solve allocates."""
    s = SCENES[name]()
    c = api.Context.from_scene(s, r_eps=0.2)
    tr = transducer(0)
    c.set_transducer(tr["centres"], tr["normals"], tr["radii"], OMEGA_RHO0)
    c.set_excitations(np.exp(2j * np.pi * np.random.default_rng(1).random((n_exc, 6))))
    kw = dict(precision=1, tol=1e-8, operator_mode=mode, batch_rhs=batch)
    est = c.estimate_solve_bytes(n_exc, **kw)
    assert c.solve(**kw)["converged"]
    used, peak = c.memory()
    assert 0 < peak <= est, (peak, est)
    c.close()


def test_budget_evicts_idle_scenes(api):
    """A budget that admits one scene's solve but not two scenes resident at
    once: requests alternating between the scenes all complete (the idle
    scene is evicted and rebuilt on its next request), the device bytes never
    pass the budget, and a rebuilt scene gives the same result."""
    probe, ids = make_server(api, ["sphere", "shell"], slots=1)
    est = [probe.estimate(ids[n], 1) for n in ("sphere", "shell")]
    probe.close()
    budget = max(est) + (1 << 20)
    srv, ids = make_server(api, ["sphere", "shell"], slots=2, hbm_budget_bytes=budget)
    w = np.exp(2j * np.pi * np.arange(6) / 6.0)[None, :]
    hs = [(name, srv.submit(ids[name], w)) for name in ["sphere", "shell"] * 3]
    for name, h in hs:
        assert srv.wait(h, 900) == 2, (srv.error(h), srv.stats(), est, budget)
    st = srv.stats()
    assert st["completed"] == 6 and st["evictions"] >= 1
    assert st["peak_device_bytes"] <= budget
    U0, _ = srv.result(hs[0][1], 1, ids["sphere"])
    U4, _ = srv.result(hs[4][1], 1, ids["sphere"])
    assert rel(U4, U0) < 1e-6
    srv.close()


def test_request_that_can_never_fit_is_refused(api):
    srv, ids = make_server(api, ["sphere"], hbm_budget_bytes=8 << 20)
    h = srv.submit(ids["sphere"], np.ones((1, 6)))
    assert srv.wait(h, 60) == 3
    with pytest.raises(Exception):
        srv.result(h, 1, ids["sphere"])
    assert srv.stats()["failed"] == 1
    srv.close()


def test_two_scenes_overlap_on_the_device(api):
    """Requests for two scenes submitted together run at the same time, each
    on its scene's own stream: the server reports two solves on the GPU at
    once, and the pair finishes clearly sooner than the same two requests run
    one after the other (the kernels of the two solves overlap)."""
    import time
    srv = api.Server(precision=1, tol=TOL, slots=2, max_batch_rhs=8, hbm_budget_bytes=8 << 30)
    ids = [srv.add_scene(scenes.sphere_scene(3), transducer=transducer(i), omega_rho0=OMEGA_RHO0, r_eps=0.2)
           for i in range(2)]
    W = [np.exp(2j * np.pi * np.random.default_rng(30 + i).random((8, 6))) for i in range(2)]
    for i in ids:  # set-up (near field, preconditioner) outside the timings
        h = srv.submit(i, W[0][:1])
        srv.wait(h)
        srv.result(h, 1, i)
    solo = []
    for k, i in enumerate(ids):
        t0 = time.perf_counter()
        h = srv.submit(i, W[k])
        srv.wait(h)
        solo.append(time.perf_counter() - t0)
        srv.result(h, 8, i)
    t0 = time.perf_counter()
    hs = [srv.submit(i, W[k]) for k, i in enumerate(ids)]
    most = 0
    while any(srv.poll(h) in (0, 1) for h in hs):  # queued or running
        most = max(most, srv.stats()["running"])
        time.sleep(0.001)
    both = time.perf_counter() - t0
    for k, (h, i) in enumerate(zip(hs, ids)):
        srv.result(h, 8, i)
    srv.close()
    print("solo", solo, "together", both, "most running", most)
    assert most == 2
    assert both < 0.85 * sum(solo)


def test_request_joins_a_running_solve(api):
    """A request for a scene whose mixed solve is already running joins it at
    its next refinement boundary instead of waiting for it to finish: the
    server counts the join, the late request is solved in the same batch
    (batch size 2 + 1), and every excitation of both requests matches the
    oracle's dense solve.  (Joining is timed against a running solve; the
    late request is submitted as soon as the first one runs, up to three
    tries.)"""
    import time
    rng = np.random.default_rng(41)
    wA = np.exp(2j * np.pi * rng.random((2, 6)))
    wB = np.exp(2j * np.pi * rng.random((1, 6)))
    for attempt in range(3):
        srv, ids = make_server(api, ["two"], slots=1, max_batch_rhs=8)
        sid = ids["two"]
        h = srv.submit(sid, wA[:1])  # set-up outside the experiment
        srv.wait(h)
        srv.result(h, 1, sid)
        hA = srv.submit(sid, wA)
        while srv.poll(hA) == 0:
            time.sleep(0.0002)
        hB = srv.submit(sid, wB)
        assert srv.wait(hA, 600) == 2 and srv.wait(hB, 600) == 2
        UA, repA = srv.result(hA, 2, sid)
        UB, repB = srv.result(hB, 1, sid)
        st = srv.stats()
        srv.close()
        if st["joined"] >= 1:
            break
    assert st["joined"] >= 1 and repB["batch_exc"] == 3 and repA["batch_exc"] == 3
    for U, W in ((UA, wA), (UB, wB)):
        for r in range(W.shape[0]):
            assert rel(U[r], oracle_solution("two", 0, W[r])) < 1e-6
