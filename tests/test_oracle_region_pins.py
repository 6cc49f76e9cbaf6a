"""Pins of the detection post-processing oracle (oracle/region.py) against
facts that do not come from it: hand-worked decode and NMS examples
(tests/golden/region_decode_hand.txt), closed forms of sigmoid, softmax and
IoU, torch's float64 sigmoid / exp / softmax over whole maps, and the
property that defines greedy NMS.  A swapped coordinate, a wrong anchor or
channel index, an unnormalised softmax or a reversed suppression order fails
at least one of them."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import region
from test_oracle_pins import _blocks

GOLD = os.path.join(os.path.dirname(__file__), "golden", "region_decode_hand.txt")


def test_decode_hand_example():
    g = _blocks(GOLD)
    fmap = g["map"].reshape(7, 1, 2)
    boxes = region.decode(fmap, [(1.0, 2.0)], 2)
    assert len(boxes) == 2
    for got, want in zip(boxes, g["boxes"]):
        x, y, w, h, obj, p = got
        np.testing.assert_allclose([x, y, w, h, obj] + p, want, rtol=1e-14, atol=1e-15)
    cand = region.candidates(boxes, 2, 0.22)
    assert [(b, round(s, 12)) for b, s, _ in cand[0]] == [(0, 0.25), (1, 0.6)]
    assert [(b, round(s, 12)) for b, s, _ in cand[1]] == [(0, 0.25)]


def test_nms_hand_example():
    g = _blocks(GOLD)
    cands = [(int(r[0]), r[1], tuple(r[2:])) for r in g["nms_in"]]
    kept = region.nms(cands, 0.45)
    assert [k[0] for k in kept] == [int(v) for v in g["nms_kept"].ravel()]
    assert region.iou(cands[0][2], cands[1][2]) == pytest.approx(0.6)
    assert region.iou(cands[0][2], cands[2][2]) == pytest.approx(1.0 / 3.0)


def test_sigmoid_softmax_closed_forms_and_torch():
    assert region.sigmoid(0.0) == 0.5
    v = np.random.default_rng(1).normal(0, 4, 200)
    for t in v:
        assert region.sigmoid(t) + region.sigmoid(-t) == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose([region.sigmoid(t) for t in v], torch.sigmoid(torch.from_numpy(v)).numpy(),
                               rtol=1e-14, atol=1e-300)
    l = list(v[:20])
    p = region.softmax(l)
    assert sum(p) == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(p, torch.softmax(torch.from_numpy(v[:20]), 0).numpy(), rtol=1e-13)
    np.testing.assert_allclose(region.softmax([t + 7.5 for t in l]), p, rtol=1e-13)   # shift invariant
    assert region.softmax([0.3] * 20) == pytest.approx([0.05] * 20)


def test_iou_closed_forms():
    a = (0.5, 0.5, 0.2, 0.4)
    assert region.iou(a, a) == pytest.approx(1.0)
    assert region.iou(a, (0.9, 0.9, 0.1, 0.1)) == 0.0
    assert region.iou((0, 0, 1, 1), (0.5, 0, 1, 1)) == pytest.approx(1.0 / 3.0)   # half overlap
    assert region.iou((0, 0, 1, 1), (0, 0, 0.5, 0.5)) == pytest.approx(0.25)      # containment
    assert region.iou((0, 0, 1, 1), (1.0, 0, 1, 1)) == 0.0                         # touching edges
    b = (0.3, 0.6, 0.5, 0.2)
    assert region.iou(a, b) == region.iou(b, a)


def _torch_decode(fmap, anchors, C):
    """Independent vectorised float64 decode with torch routines."""
    t = torch.from_numpy(np.asarray(fmap, np.float64))
    A = len(anchors)
    ch, GH, GW = t.shape
    t = t.reshape(A, 5 + C, GH, GW)
    jj = torch.arange(GW, dtype=torch.float64)[None, None, :]
    ii = torch.arange(GH, dtype=torch.float64)[None, :, None]
    pw = torch.tensor([a[0] for a in anchors], dtype=torch.float64)[:, None, None]
    ph = torch.tensor([a[1] for a in anchors], dtype=torch.float64)[:, None, None]
    x = (jj + torch.sigmoid(t[:, 0])) / GW
    y = (ii + torch.sigmoid(t[:, 1])) / GH
    w = torch.exp(t[:, 2]) * pw / GW
    h = torch.exp(t[:, 3]) * ph / GH
    obj = torch.sigmoid(t[:, 4])
    p = torch.softmax(t[:, 5:], dim=1)
    # box id (i*GW + j)*A + a: order axes (GH, GW, A)
    stack = torch.stack([x, y, w, h, obj], dim=-1).permute(1, 2, 0, 3).reshape(-1, 5)
    probs = p.permute(2, 3, 0, 1).reshape(-1, C)
    return stack.numpy(), probs.numpy()


ANCH = [(0.8, 1.2), (2.0, 3.1), (4.5, 2.2), (6.0, 7.5), (9.7, 5.0)]


def test_decode_vs_torch_on_random_maps():
    rng = np.random.default_rng(7)
    for GH, GW, C in ((13, 13, 20), (5, 9, 3)):
        fmap = rng.normal(0, 2, (len(ANCH) * (5 + C), GH, GW))
        got = region.decode(fmap, ANCH, C)
        st, pr = _torch_decode(fmap, ANCH, C)
        np.testing.assert_allclose(np.array([g[:5] for g in got]), st, rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(np.array([g[5] for g in got]), pr, rtol=1e-12, atol=1e-300)


def test_nms_defining_property_on_random_candidates():
    """Greedy NMS is the one set where a candidate is kept exactly when no
    kept candidate ranked before it overlaps it above the threshold."""
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(1, 60))
        cands = [(i, float(rng.choice([0.3, 0.5, rng.random()])),
                  (rng.random(), rng.random(), 0.05 + 0.3 * rng.random(), 0.05 + 0.3 * rng.random()))
                 for i in range(n)]
        thr = float(rng.uniform(0.2, 0.7))
        kept = region.nms(cands, thr)
        keep_ids = {k[0] for k in kept}
        order = sorted(cands, key=lambda t: (-t[1], t[0]))
        for r, c in enumerate(order):
            earlier_kept = [o for o in order[:r] if o[0] in keep_ids]
            should = all(region.iou(c[2], o[2]) <= thr for o in earlier_kept)
            assert (c[0] in keep_ids) == should
        # kept ones come out in rank order
        ranks = {c[0]: r for r, c in enumerate(order)}
        assert [ranks[k[0]] for k in kept] == sorted(ranks[k[0]] for k in kept)


def test_detect_groups_by_class_and_truncates():
    rng = np.random.default_rng(11)
    C = 4
    fmaps = rng.normal(0, 2, (2, len(ANCH) * (5 + C), 6, 7))
    res = region.detect(fmaps, ANCH, C, 0.1, 0.45, 5)
    full = region.detect(fmaps, ANCH, C, 0.1, 0.45, 10 ** 6)
    for (n, d), (n2, d2) in zip(res, full):
        assert n == n2 == len(d2) and d == d2[:5]
        assert [t[0] for t in d2] == sorted(t[0] for t in d2)       # class order
        for c in range(C):
            s = [t[2] for t in d2 if t[0] == c]
            assert s == sorted(s, reverse=True)
