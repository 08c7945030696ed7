"""Sub-block construction from the visibility graph (Sec. 5.2), rpba_partition:
a host function of the library (no GPU). Checked against brute force (node
weights, edge cut), for balance, connectivity and determinism, against the
hand-made partition of the 1,000-camera block, and by running the method on
its sub-blocks."""

import itertools
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1910_08138_gb300 import rpba, synth  # noqa: E402


def brute_graph(prob):
    """Node weights (cube root of the summed observation counts of the points a
    camera sees) and edges {(a, b): shared points}, by direct counting."""
    oc, op = np.asarray(prob["obs_cam"]), np.asarray(prob["obs_point"])
    M = prob["cam_pose"].shape[0]
    n_obs = np.bincount(op, minlength=prob["points"].shape[0])
    w = np.cbrt(np.bincount(oc, weights=n_obs[op], minlength=M))
    edges = {}
    order = np.argsort(op, kind="stable")
    for cams in np.split(oc[order], np.flatnonzero(np.diff(op[order])) + 1):
        for a, b in itertools.combinations(np.unique(cams), 2):
            edges[(a, b)] = edges.get((a, b), 0) + 1
    return w, edges


def cut_of(edges, part):
    return sum(c for (a, b), c in edges.items() if part[a] != part[b])


def partition(prob, L):
    return rpba.rpba_partition(prob["cam_pose"].shape[0], prob["points"].shape[0], prob["obs_cam"],
                               prob["obs_point"], L)


@pytest.fixture(scope="module")
def block1000():
    prob = synth.config(2)
    return prob, brute_graph(prob)


def test_weights_and_cut_against_brute_force(block1000):
    prob, (w_ref, edges) = block1000
    part, w, cut = partition(prob, 8)
    np.testing.assert_allclose(w, w_ref, rtol=1e-14)
    assert cut == cut_of(edges, part)


def test_balance_connectivity_and_a_smaller_cut_than_the_hand_made_runs(block1000):
    prob, (w_ref, edges) = block1000
    L = 8
    part, w, cut = partition(prob, L)
    W = np.bincount(part, weights=w, minlength=L)
    assert np.all(W > 0)
    # each bisection keeps a side within 2 % of its share: three levels
    assert W.max() / W.mean() <= 1.03 ** 3 and W.min() / W.mean() >= 0.97 ** 3
    # every sub-block is connected in the visibility graph
    adj = {}
    for (a, b) in edges:
        adj.setdefault(a, []).append(b)
        adj.setdefault(b, []).append(a)
    for l in range(L):
        cams = set(np.flatnonzero(part == l).tolist())
        seen, stack = set(), [next(iter(cams))]
        while stack:
            u = stack.pop()
            if u in seen:
                continue
            seen.add(u)
            stack.extend(v for v in adj.get(u, []) if v in cams)
        assert seen == cams, l
    # fewer shared points between sub-blocks (fewer TPs to exchange) than the
    # eight contiguous column runs the benchmark block comes with
    assert cut < 0.6 * cut_of(edges, np.asarray(prob["cam_subblock"]))
    # deterministic
    part2, _, cut2 = partition(prob, L)
    np.testing.assert_array_equal(part, part2)
    assert cut2 == cut


def test_rejects_bad_arguments():
    prob = synth.tiny(seed=1, runs=[3, 3])
    M, N = prob["cam_pose"].shape[0], prob["points"].shape[0]
    for L in (0, M + 1):
        with pytest.raises(rpba.RpbaError) as e:
            partition(prob, L)
        assert e.value.status == 1
    bad = np.asarray(prob["obs_cam"]).copy()
    bad[0] = M
    with pytest.raises(rpba.RpbaError):
        rpba.rpba_partition(M, N, bad, prob["obs_point"], 2)
    part, _, _ = partition(prob, M)  # one camera per part
    assert sorted(part.tolist()) == list(range(M))


def test_the_method_on_its_own_sub_blocks():
    """The 50-camera block split into 2 sub-blocks by the partitioner instead
    of the grid halves: the run still ends at the noise level."""
    prob = dict(synth.config(1))
    part, _, _ = partition(prob, 2)
    prob["cam_subblock"] = part
    rep = oracle.Oracle(prob).run(robust=1, robust_from_start=1)
    assert 0.45 < rep["sigma0"] < 0.55
