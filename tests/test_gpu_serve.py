"""Serving loop: requests admitted by a device-memory budget with continuous batching. Each
request's result must match the oracle's run of the same solve (criteria in tests/_parity.py)
and be bit-identical alone and in the mix (local-stencil requests share the
batched persistent launch; RBF-PU requests run on their own streams), and admission must keep
the charged bytes within the budget."""
import math
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

import _parity  # noqa: E402

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(11)
    specs = [  # N, n, ell, power, method, mode, precision, velocity kind, T, steps
        (642, 31, 2, 5, rbfsl.LOCAL, rbfsl.DIRECT, rbfsl.FP64, 0, 2, 8),
        (1000, 55, 3, 7, rbfsl.LOCAL, rbfsl.CENTER, rbfsl.MIXED, 1, 3, 5),
        (2562, 60, 3, 7, rbfsl.PU, rbfsl.DIRECT, rbfsl.FP64, 0, 2, 6),
        (2562, 31, 2, 5, rbfsl.LOCAL, rbfsl.DIRECT, rbfsl.MIXED, 1, 1, 12),
        (1500, 84, 4, 9, rbfsl.LOCAL, rbfsl.DIRECT, rbfsl.FP64, 0, 2, 4),
        (1000, 60, 3, 7, rbfsl.PU, rbfsl.DIRECT, rbfsl.MIXED, 1, 1, 5),
    ]
    out = []
    for k, (N, n, ell, p, method, mode, prec, vk, T, steps) in enumerate(specs):
        X = inputs.nodes(N, 300 + k)
        vp = (inputs.rigid_rotation_params(inputs.random_unit_vectors(1, rng)[0], 1.0) if vk == 0
              else inputs.deformation_params(2.0, 1.0))
        tr = inputs.config_local_deformation(N=N, n_random=T).tracers
        q0fn = lambda P, tr=tr, T=T: tr(P)[:, :T]  # noqa: E731
        C = inputs.fibonacci_nodes(math.ceil(2.5 * N / n)) if method == rbfsl.PU else None
        out.append(dict(X=X, q0=q0fn(X), q0fn=q0fn, n=n, ell=ell, power=p, vel_kind=vk, vel_params=vp,
                        dt=1 / 40, steps=steps, method=method, mode=mode, precision=prec, centers=C))
    return out


def _submit(srv, r):
    return srv.submit(r["X"], r["q0"], r["n"], r["ell"], r["power"], r["vel_kind"], r["vel_params"],
                      r["dt"], r["steps"], method=r["method"], mode=r["mode"], precision=r["precision"],
                      centers=r["centers"])


def test_results_identical_alone_and_in_the_mix():
    reqs = _requests()
    srv = rbfsl.Server(0, budget_bytes=40 * 10 ** 9, max_slots=8)
    tickets = []
    for r in reqs:  # staggered arrivals while earlier requests are running
        tickets.append(_submit(srv, r))
        time.sleep(0.003)
    srv.wait_idle(300)
    mixed = []
    for t in tickets:
        q, st = srv.result(t)
        assert st.status == 0 and st.finish_s >= st.admit_s >= st.submit_s and st.failed_points == 0
        mixed.append(q)
    assert srv.info().ticks >= max(r["steps"] for r in reqs)
    srv.close()
    for r, qm in zip(reqs, mixed):
        alone = rbfsl.Server(0, budget_bytes=40 * 10 ** 9, max_slots=8)
        t = _submit(alone, r)
        alone.wait_idle(300)
        qa, st = alone.result(t)
        assert st.steps == r["steps"]
        np.testing.assert_array_equal(qm, qa)
        alone.close()


def test_budget_admission_and_refusal():
    reqs = [r for r in _requests() if r["method"] == rbfsl.LOCAL]
    srv = rbfsl.Server(0, budget_bytes=10 ** 9, max_slots=64)
    tickets = [_submit(srv, r) for r in reqs]
    srv.wait_idle(300)
    charged = []
    for t in tickets:
        _, st = srv.result(t)
        assert st.status == 0
        charged.append(st.device_bytes)
    info = srv.info()
    assert info.peak_bytes <= info.budget_bytes and info.used_bytes == 0
    srv.close()
    # a budget smaller than every request: each runs alone, one after the other
    small = rbfsl.Server(0, budget_bytes=max(charged) + 1, max_slots=64)
    tickets = [_submit(small, r) for r in reqs]
    small.wait_idle(300)
    stats = [small.result(t)[1] for t in tickets]
    assert all(s.status == 0 for s in stats)
    for a in stats:  # requests that ran at the same time fit the budget together
        for b in stats:
            if a is not b and a.admit_s < b.finish_s and b.admit_s < a.finish_s:
                assert a.device_bytes + b.device_bytes <= max(charged) + 1
    assert small.info().peak_bytes <= max(charged) + 1
    small.close()
    tiny = rbfsl.Server(0, budget_bytes=1000, max_slots=4)
    with pytest.raises(rbfsl.RbfslError) as e:
        _submit(tiny, reqs[0])
    assert e.value.code == rbfsl.ENOMEM
    tiny.close()


def _oracle_run(orc, r):
    if r["method"] == rbfsl.LOCAL:
        return orc.local_run(r["X"], r["q0"], r["n"], r["ell"], r["power"], r["vel_kind"], r["vel_params"],
                             r["dt"], r["steps"], mode=r["mode"])
    pu = orc.PUInterpolator(r["X"], r["centers"], r["n"], r["ell"], r["power"])
    q = r["q0"]
    for m in range(r["steps"]):
        q = pu.apply(orc.trace_rk4(r["X"], r["vel_kind"], r["vel_params"], (m + 1) * r["dt"], r["dt"]), q)
    return q


def test_served_results_match_oracle(orc):
    """Every request of the mix (local direct / centre stencils and RBF-PU, FP64 and mixed)
    served together, each against the oracle's run of the same solve."""
    reqs = _requests()
    srv = rbfsl.Server(0, budget_bytes=40 * 10 ** 9, max_slots=8)
    tickets = []
    for r in reqs:
        tickets.append(_submit(srv, r))
        time.sleep(0.003)
    srv.wait_idle(300)
    got = [srv.result(t)[0] for t in tickets]
    srv.close()
    for k, (r, g) in enumerate(zip(reqs, got)):
        ref = _oracle_run(orc, r)
        ex = _parity.exact_field(r["q0fn"], r["X"], r["vel_kind"], r["vel_params"], r["steps"] * r["dt"])
        strict = r["precision"] == rbfsl.FP64 and r["method"] == rbfsl.LOCAL and r["n"] == 31
        _parity.check_run(f"served[{k}] method={r['method']} N={r['X'].shape[0]} n={r['n']} "
                          f"prec={r['precision']}", g, ref, ex, strict)


def test_served_centre_class_mix():
    """The served workload's shape at small sizes: local centre-stencil requests of all three
    (n, ell) classes at once (each its own persistent launch on a parallel graph branch), RBF-PU
    requests on their own streams, 1 to 16 tracers, mixed precision and FP64, staggered arrivals:
    every request must finish with status 0, no failed point and a finite field."""
    rng = np.random.default_rng(23)
    reqs = []
    classes = [(31, 2, 5), (55, 3, 7), (84, 4, 9)]
    for k in range(15):
        N = [642, 2562, 10242][k % 3]
        T = [1, 7, 16, 3, 11][k % 5]
        X = inputs.nodes(N, 700 + k)
        vp = inputs.rigid_rotation_params(inputs.random_unit_vectors(1, rng)[0], 1.0)
        tr = inputs.config_local_deformation(N=N, n_random=T).tracers
        q0 = tr(X)[:, :T]
        if k % 5 == 4:
            n, ell, p, method, mode = 60, 3, 7, rbfsl.PU, rbfsl.DIRECT
            C = inputs.fibonacci_nodes(math.ceil(2.5 * N / n))
        else:
            (n, ell, p), method, mode, C = classes[k % 3], rbfsl.LOCAL, rbfsl.CENTER, None
        prec = rbfsl.FP64 if k % 4 == 3 else rbfsl.MIXED
        reqs.append(dict(X=X, q0=q0, n=n, ell=ell, power=p, vel_kind=0, vel_params=vp, dt=1 / 30,
                         steps=6 + k % 4, method=method, mode=mode, precision=prec, centers=C))
    srv = rbfsl.Server(0, budget_bytes=40 * 10 ** 9, max_slots=16)
    tickets = []
    for r in reqs:
        tickets.append(_submit(srv, r))
        time.sleep(0.002)
    srv.wait_idle(600)
    for r, t in zip(reqs, tickets):
        q, st = srv.result(t, raise_on_failure=False)
        assert st.status == 0, st.message.decode()
        assert st.steps == r["steps"] and st.failed_points == 0
        assert q is not None and np.isfinite(q).all()
    srv.close()
