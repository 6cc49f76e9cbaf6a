"""FP64 oracle of the detection post-processing after the last conv layer.

TEST INFRASTRUCTURE ONLY (see the package docstring): tests/, the smoke check
and bench.py's CPU-baseline leg are its only users.

The paper offloads Darknet's "detection" sample app (Sec. 5.1.1) and prints
none of its steps.  What follows is the plain definition of the region
(anchor-box) output of a Darknet detection network, written out in FP64 with
Python loops:

* The final map has A * (5 + C) channels over a GH x GW grid.  Anchor a owns
  channels a*(5+C) .. a*(5+C)+4+C: tx, ty, tw, th, to, then C class logits.
* Cell (i, j) (row i, column j) and anchor a form box id (i*GW + j)*A + a:
    x = (j + sigmoid(tx)) / GW,        y = (i + sigmoid(ty)) / GH,
    w = exp(tw) * pw / GW,             h = exp(th) * ph / GH,
  (x, y) the centre and (w, h) the size as fractions of the frame, (pw, ph)
  the anchor's prior in grid cells.
* objectness = sigmoid(to); class probabilities = softmax of the C logits;
  the class-c score is objectness * p_c.  A box is a candidate of class c
  when its class-c score exceeds the score threshold.
* Greedy non-maximum suppression per class: candidates taken in order of
  score (descending; equal scores by id, ascending); a candidate is kept
  unless its intersection-over-union with a box already kept for the class
  exceeds the IoU threshold.
* A frame's detections: its kept boxes, class by class (ascending), each
  class in the order above; at most max_det of them are reported, and the
  count is the number kept before that cut.
"""
from __future__ import annotations

import math

import numpy as np


def sigmoid(v: float) -> float:
    return 1.0 / (1.0 + math.exp(-v))


def softmax(logits):
    m = max(logits)
    e = [math.exp(v - m) for v in logits]
    s = sum(e)
    return [t / s for t in e]


def iou(a, b) -> float:
    """IoU of two (x, y, w, h) centre-size boxes."""
    al, ar, at, ab = a[0] - a[2] / 2, a[0] + a[2] / 2, a[1] - a[3] / 2, a[1] + a[3] / 2
    bl, br, bt, bb = b[0] - b[2] / 2, b[0] + b[2] / 2, b[1] - b[3] / 2, b[1] + b[3] / 2
    iw = min(ar, br) - max(al, bl)
    ih = min(ab, bb) - max(at, bt)
    inter = max(iw, 0.0) * max(ih, 0.0)
    union = a[2] * a[3] + b[2] * b[3] - inter
    return inter / union if union > 0 else 0.0


def decode(fmap, anchors, n_classes: int):
    """All boxes of one frame's map (A*(5+C), GH, GW): list indexed by box
    id of (x, y, w, h, objectness, [p_0 .. p_{C-1}])."""
    fmap = np.asarray(fmap, dtype=np.float64)
    A = len(anchors)
    C = n_classes
    ch, GH, GW = fmap.shape
    assert ch == A * (5 + C)
    out = []
    for i in range(GH):
        for j in range(GW):
            for a in range(A):
                base = a * (5 + C)
                tx, ty, tw, th, to = (float(fmap[base + k, i, j]) for k in range(5))
                pw, ph = anchors[a]
                x = (j + sigmoid(tx)) / GW
                y = (i + sigmoid(ty)) / GH
                w = math.exp(tw) * pw / GW
                h = math.exp(th) * ph / GH
                p = softmax([float(fmap[base + 5 + c, i, j]) for c in range(C)])
                out.append((x, y, w, h, sigmoid(to), p))
    return out


def candidates(boxes, n_classes: int, score_thresh: float):
    """Per class: list of (id, score, (x, y, w, h)) with score > threshold."""
    cand = [[] for _ in range(n_classes)]
    for bid, (x, y, w, h, obj, p) in enumerate(boxes):
        for c in range(n_classes):
            s = obj * p[c]
            if s > score_thresh:
                cand[c].append((bid, s, (x, y, w, h)))
    return cand


def nms(cands, iou_thresh: float):
    """Greedy NMS of one class's candidates; returns the kept ones in order."""
    order = sorted(cands, key=lambda t: (-t[1], t[0]))
    kept = []
    for bid, s, box in order:
        if all(iou(box, k[2]) <= iou_thresh for k in kept):
            kept.append((bid, s, box))
    return kept


def detect(fmaps, anchors, n_classes: int, score_thresh: float, iou_thresh: float, max_det: int):
    """Detections of each frame of an (N, A*(5+C), GH, GW) map: per frame
    (count, [(cls, id, score, x, y, w, h), ...] of at most max_det)."""
    res = []
    for f in np.asarray(fmaps, dtype=np.float64):
        cand = candidates(decode(f, anchors, n_classes), n_classes, score_thresh)
        dets = []
        for c in range(n_classes):
            for bid, s, box in nms(cand[c], iou_thresh):
                dets.append((c, bid, s) + tuple(box))
        res.append((len(dets), dets[:max_det]))
    return res
