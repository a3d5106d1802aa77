"""The differentiation path: expected counts of a REAL graph as a function of
the probabilities p it is given (torch.autograd), their hand-written adjoint,
and ubt_set_edge_values, which loads a new p into a built graph.

Pinned against the oracle's analytic gradient (the term-wise derivative of
Sec. 3's four-term P_bal sum) and against difference quotients of the GPU's
own forward.  E is affine in each p_e (the three edges of a triangle are
distinct, so p_e enters every P_bal at most linearly), so the central
difference at p_e = 1/2 with step h = 1/2,

    (E(p_e = 1) - E(p_e = 0)) / 1,

is the derivative exactly.  Its endpoints 0 and 1 are stored exactly by the
graph (s = 1 - 2p = -1, +1), so the quotient carries only the forward's own
rounding (2^-31 per triangle product), far below the tolerance; a small step
such as 10^-3 would divide that rounding by 2 * 10^-3.

Tolerance (gradient, per edge): |g - g_ref| <= 1e-5 max(|g_ref|, 1e-3 A_e),
A_e = sum over the edge's triangles of |(1 - 2p_f)(1 - 2p_g)| (the floor is
used where the terms cancel); expected counts within 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import difference_quotients, grad_report, mixed_graph, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ubt():
    return require_gpu()


def test_forward_and_backward_follow_p_updated_in_place(ubt):
    """p changed in place twice after the build: every forward and backward
    answers for the current p, without a rebuild."""
    import torch
    n, m = 3000, 40000
    s, d = mixed_graph(n, m, 21)
    p0 = synth.p_uniform_f32(s.size, 22)
    pt = torch.from_numpy(p0.copy()).cuda().requires_grad_(True)
    G = ubt.Graph(n, s, d, p=pt.detach())
    rng = synth.rng(23)
    for step in range(3):
        if step:
            with torch.no_grad():  # an optimiser-style in-place update
                pt.copy_(torch.from_numpy(rng.random(s.size).astype(np.float32)).cuda())
        p = pt.detach().cpu().numpy()
        pt.grad = None
        eb, eu = ubt.expected_counts(G, pt)
        ob, ou, _ = oracle.expected_real(n, s, d, p)
        assert abs(eb.item() - ob) <= 1e-9 * max(1.0, abs(ob)), step
        assert abs(eu.item() - ou) <= 1e-9 * max(1.0, abs(ou)), step
        eb.backward()
        og, ga = oracle.grad_real(n, s, d, p, with_abs=True)
        ok, rel, floored = grad_report(pt.grad.double().cpu().numpy(), og, ga)
        assert ok.all(), (step, int((~ok).sum()))
    assert G.guard() == 0


def test_backward_uses_the_p_of_its_own_forward(ubt):
    """Two forwards at different p, then the first one's backward: the adjoint
    reloads the p saved by its forward."""
    import torch
    s, d = synth.er_graph(1500, 15000, 31)
    pa = torch.from_numpy(synth.p_uniform_f32(s.size, 32)).cuda().requires_grad_(True)
    pb = torch.from_numpy(synth.p_uniform_f32(s.size, 33)).cuda().requires_grad_(True)
    G = ubt.Graph(1500, s, d, p=pa.detach())
    ea, _ = ubt.expected_counts(G, pa)
    eb_, _ = ubt.expected_counts(G, pb)
    ea.backward()
    og, ga = oracle.grad_real(1500, s, d, pa.detach().cpu().numpy(), with_abs=True)
    ok, _, _ = grad_report(pa.grad.double().cpu().numpy(), og, ga)
    assert ok.all()
    ob, _, _ = oracle.expected_real(1500, s, d, pb.detach().cpu().numpy())
    assert abs(eb_.item() - ob) <= 1e-9 * max(1.0, abs(ob))


def test_set_edge_values_rejects_out_of_range_entries(ubt):
    """An entry outside [0, 1] keeps its old value and is reported by the
    self-check word (code 6, detail = its input index)."""
    import torch
    s, d = synth.er_graph(500, 4000, 41)
    p = synth.p_uniform_f32(s.size, 42)
    G = ubt.Graph(500, s, d, p=torch.from_numpy(p).cuda())
    e0 = G.expected_counts()
    bad = torch.from_numpy(p.copy()).cuda()
    bad[17] = 1.5
    bad[5] = float("nan")
    G.set_edge_values_(bad)
    w = G.guard()
    assert (w >> 56) == 6 and (w & ((1 << 56) - 1)) in (5, 17)
    good = p.copy()
    ob, _, _ = oracle.expected_real(500, s, d, good)
    # every other entry took its (unchanged) value; the two bad ones kept theirs
    assert abs(G.expected_counts()[0] - ob) <= 1e-9 * max(1.0, abs(ob))
    assert abs(e0[0] - ob) <= 1e-9 * max(1.0, abs(ob))
    Gk = ubt.Graph(500, s, d, k=synth.k_uniform(s.size, 43))
    with pytest.raises(ubt.UbtError):
        Gk.set_edge_values_(torch.from_numpy(p).cuda())


def test_gradient_against_difference_quotients_small(ubt):
    import torch
    s, d = mixed_graph(400, 3000, 51)
    p = synth.p_uniform_f32(s.size, 52)
    pt = torch.from_numpy(p.copy()).cuda().requires_grad_(True)
    G = ubt.Graph(400, s, d, p=pt.detach())
    eb, _ = ubt.expected_counts(G, pt)
    eb.backward()
    got = pt.grad.double().cpu().numpy()
    fd = difference_quotients(ubt, G, p, np.arange(s.size))
    _, ga = oracle.grad_real(400, s, d, p, with_abs=True)
    ok, rel, floored = grad_report(got, fd, ga)
    assert ok.all(), (int((~ok).sum()), float(rel[~ok].max()))
    assert G.guard() == 0
