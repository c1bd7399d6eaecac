"""Batched local RBF-SL (many problems, one persistent fused kernel per step, CUDA graph):
every problem's result must match the oracle's run of the same problem (Algorithm 1; criteria
in tests/_parity.py), and be bit-identical to the same problem stepped alone and to the
single-problem context path, with or without the graph, before and after autotuning, and
while other problems are added and removed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

import _parity  # noqa: E402

pytestmark = pytest.mark.gpu


def _problems():
    rng = np.random.default_rng(7)
    specs = [  # N, n, ell, power, mode, precision, velocity, T
        (642, 31, 2, 5, rbfsl.DIRECT, rbfsl.FP64, 0, 1),
        (1000, 55, 3, 7, rbfsl.DIRECT, rbfsl.MIXED, 1, 3),
        (1500, 84, 4, 9, rbfsl.DIRECT, rbfsl.FP64, 0, 5),
        (2562, 31, 2, 5, rbfsl.CENTER, rbfsl.FP64, 1, 2),
        (777, 55, 3, 7, rbfsl.CENTER, rbfsl.MIXED, 0, 4),
        (900, 84, 4, 9, rbfsl.DIRECT, rbfsl.MIXED, 1, 2),
        (1200, 84, 4, 9, rbfsl.CENTER, rbfsl.FP64, 0, 2),
    ]
    out = []
    for k, (N, n, ell, p, mode, prec, vk, T) in enumerate(specs):
        X = inputs.nodes(N, 100 + k)
        if vk == 0:
            vp = inputs.rigid_rotation_params(inputs.random_unit_vectors(1, rng)[0], rng.uniform(0.5, 2.0))
        else:
            vp = inputs.deformation_params(rng.uniform(1.5, 2.5), 1.0)
        tr = inputs.config_local_deformation(N=N, n_random=T).tracers
        q0fn = lambda P, tr=tr, T=T: tr(P)[:, :T]  # noqa: E731
        out.append(dict(X=X, q0=q0fn(X), q0fn=q0fn, n=n, ell=ell, power=p, mode=mode, precision=prec, vk=vk,
                        vp=vp, dt=1.0 / 50))
    return out


def _add(b, P):
    return b.add(P["X"], P["q0"], P["n"], P["ell"], P["power"], P["vk"], P["vp"], P["dt"],
                 mode=P["mode"], precision=P["precision"])


def _ctx(P, steps):
    c = rbfsl.Context(0)
    c.set_nodes(P["X"])
    c.set_velocity(P["vk"], P["vp"])
    c.set_method(rbfsl.LOCAL, P["mode"])
    c.set_stencil_size(P["n"])
    c.set_sh_degree(P["ell"])
    c.set_kernel(rbfsl.PHS, P["power"])
    c.set_precision(P["precision"])
    c.set_dt(P["dt"])
    c.set_tracers(P["q0"])  # FP64 in both precisions: mixed stores it as FP32 pairs, like the batch
    c.step(steps)
    out = c.get_q()
    c.close()
    return out


def test_batch_equals_context_and_alone_bitwise():
    probs = _problems()
    S = 6
    s = torch.cuda.Stream()
    b = rbfsl.Batch(0, stream=s)
    ids = [_add(b, P) for P in probs]
    b.step(S)
    got = [b.get_q(i) for i in ids]
    for i in ids:
        st = b.stats(i)
        assert st.steps_done == S and st.singular_points == 0 and st.knn_failures == 0
    b.close()
    for P, g in zip(probs, got):
        np.testing.assert_array_equal(g, _ctx(P, S))
    alone = rbfsl.Batch(0, stream=s)
    pid = _add(alone, probs[2])
    alone.step(S)
    np.testing.assert_array_equal(alone.get_q(pid), got[2])
    alone.close()


def test_batch_graph_eager_autotune_and_membership_changes():
    probs = _problems()
    s = torch.cuda.Stream()
    b1 = rbfsl.Batch(0, stream=s)
    b2 = rbfsl.Batch(0, stream=s)
    b2.set_graph(False)
    ids1 = [_add(b1, P) for P in probs[:4]]
    ids2 = [_add(b2, P) for P in probs[:4]]
    b1.step(2)
    b2.step(2)
    choices = b1.autotune()
    assert {(n, ell) for n, ell, _ in choices} == {(31, 2), (55, 3), (84, 4)}
    b1.step(2)
    b2.step(2)
    for i1, i2 in zip(ids1, ids2):
        np.testing.assert_array_equal(b1.get_q(i1), b2.get_q(i2))
    # a problem leaves and two join while the others keep stepping
    b1.remove(ids1[1])
    new = [_add(b1, probs[4]), _add(b1, probs[5])]
    b1.step(3)
    np.testing.assert_array_equal(b1.get_q(ids1[0]), _ctx(probs[0], 7))
    np.testing.assert_array_equal(b1.get_q(ids1[3]), _ctx(probs[3], 7))
    np.testing.assert_array_equal(b1.get_q(new[0]), _ctx(probs[4], 3))
    np.testing.assert_array_equal(b1.get_q(new[1]), _ctx(probs[5], 3))
    b1.close()
    b2.close()


def test_batch_matches_oracle(orc):
    """Every problem of the batch (n = 31 / 55 / 84, direct and centre stencils, FP64 and
    mixed, rotation and deformation) against the oracle's run of Algorithm 1."""
    probs = _problems()
    S = 6
    s = torch.cuda.Stream()
    b = rbfsl.Batch(0, stream=s)
    ids = [_add(b, P) for P in probs]
    b.step(S)
    got = [b.get_q(i) for i in ids]
    b.close()
    for k, (P, g) in enumerate(zip(probs, got)):
        ref = orc.local_run(P["X"], P["q0"], P["n"], P["ell"], P["power"], P["vk"], P["vp"], P["dt"], S,
                            mode=P["mode"])
        ex = _parity.exact_field(P["q0fn"], P["X"], P["vk"], P["vp"], S * P["dt"])
        strict = P["precision"] == rbfsl.FP64 and P["n"] == 31
        _parity.check_run(f"batch[{k}] N={P['X'].shape[0]} n={P['n']} mode={P['mode']} prec={P['precision']}",
                          g, ref, ex, strict)
