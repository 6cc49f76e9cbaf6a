"""Detection post-processing on the GPU (net_set_region / net_detect_device /
net_forward_detect) against the FP64 oracle (oracle/region.py).

The kernels decide in FP32 which boxes pass the score threshold and which
suppress which; the oracle decides in FP64.  So the comparison has two
parts: what is unique (each detection's decoded box and score, matched by
(class, id), to 5e-6) and, for the kept sets, validity checked with the
oracle's own FP64 boxes: every kept box scores above the threshold, no two
kept boxes of a class overlap beyond the IoU threshold, every candidate
left out is suppressed by a kept box ranked before it; any set difference
must come from a decision within 1e-5 of a threshold."""
import numpy as np
import pytest

import oracle
from oracle import region
from paper_1811_03882_gb300 import synth
from helpers import make_net

pytestmark = pytest.mark.gpu
ANCH = [(0.8, 1.2), (2.0, 3.1), (4.5, 2.2), (6.0, 7.5), (9.7, 5.0)]
C = 20
BAND = 1e-5     # decisions this close to a threshold may go either way


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def _check_frame(fmap, cnt, dets, thr, nms_thr, max_det, anch=ANCH, C=C):
    """One frame's GPU detections against the oracle decode of the same map."""
    boxes = region.decode(fmap, anch, C)
    ref_n, ref = region.detect(fmap[None], anch, C, thr, nms_thr, 10 ** 6)[0]
    got = [(int(d["cls"]), int(d["id"]), float(d["score"]), float(d["x"]), float(d["y"]), float(d["w"]),
            float(d["h"])) for d in dets[:min(cnt, max_det)]]
    # the reported rows: class order, score order within a class (ties by id)
    key = [(g[0], -g[2], g[1]) for g in got]
    assert key == sorted(key)
    # unique parts: each reported box's decode and score
    for c, bid, s, x, y, w, h in got:
        bx, by, bw, bh, obj, p = boxes[bid]
        np.testing.assert_allclose([s, x, y, w, h], [obj * p[c], bx, by, bw, bh], rtol=5e-6, atol=1e-7)
    if cnt > max_det:
        return cnt, ref_n, 0
    # validity of the kept sets, in FP64 with the oracle's boxes
    kept = {(g[0], g[1]) for g in got}
    diff = kept ^ {(r[0], r[1]) for r in ref}
    for c in range(C):
        kc = [bid for (cc, bid) in kept if cc == c]
        for bid in kc:
            assert boxes[bid][4] * boxes[bid][5][c] > thr - BAND
        for a_ in range(len(kc)):
            for b_ in range(a_ + 1, len(kc)):
                assert region.iou(boxes[kc[a_]][:4], boxes[kc[b_]][:4]) <= nms_thr + BAND
        for bid, (x, y, w, h, obj, p) in enumerate(boxes):
            s = obj * p[c]
            if s > thr + BAND and bid not in kc:
                assert any(region.iou((x, y, w, h), boxes[k][:4]) > nms_thr - BAND and
                           boxes[k][4] * boxes[k][5][c] >= s - BAND for k in kc), (c, bid)
    for (c, bid) in diff:   # a set difference needs a near-threshold decision
        s = boxes[bid][4] * boxes[bid][5][c]
        near_thr = abs(s - thr) <= BAND
        near_iou = any(abs(region.iou(boxes[bid][:4], boxes[o][:4]) - nms_thr) <= BAND
                       for (cc, o) in kept | {(r[0], r[1]) for r in ref} if cc == c and o != bid)
        assert near_thr or near_iou, (c, bid, s)
    assert cnt == len(got)
    return cnt, ref_n, len(diff)


def _run_maps(maps, thr, nms_thr, max_det, anch=ANCH, C=C):
    import torch
    n, ch, gh, gw = maps.shape
    spec = synth.NetSpec("head", 8, [synth.Layer(1, ch, False, synth.ACT_LINEAR, synth.POOL_NONE)])
    with make_net(spec, prec="fp32", max_batch=n, max_side=max(gh, gw)) as net:
        net.set_region(anch, C, thr, nms_thr, max_det)
        d_map = torch.from_numpy(maps).cuda()
        d_cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        d_det = torch.zeros(n * max_det * 32, dtype=torch.uint8, device="cuda")
        net.detect_device(d_map, n, gh, gw, d_cnt, d_det)
        torch.cuda.synchronize()
        from paper_1811_03882_gb300.binding import DETECTION
        det = d_det.cpu().numpy().view(DETECTION).reshape(n, max_det)
        return d_cnt.cpu().numpy(), det


# grids of 245, 385, 845, 1805 and 3920 boxes: every size of the NMS sort
# (256, 512, 1024, 2048 and 4096 slots)
@pytest.mark.parametrize("thr,nms_thr,gh,gw", [(0.05, 0.45, 13, 13), (0.2, 0.3, 19, 19), (0.01, 0.6, 7, 11),
                                              (0.03, 0.5, 7, 7), (0.25, 0.45, 28, 28)])
def test_detect_random_maps_vs_oracle(thr, nms_thr, gh, gw):
    rng = np.random.default_rng(int(thr * 1000) + gh)
    maps = rng.normal(0, 2, (3, len(ANCH) * (5 + C), gh, gw)).astype(np.float32)
    cnt, det = _run_maps(maps, thr, nms_thr, 4096)
    tot = 0
    for f in range(maps.shape[0]):
        n, ref_n, nd = _check_frame(maps[f].astype(np.float64), int(cnt[f]), det[f], thr, nms_thr, 4096)
        print("frame %d: %d kept (oracle %d), %d near-threshold differences" % (f, n, ref_n, nd))
        tot += n
    assert tot > 10


def test_detect_many_classes():
    """40 classes (beyond the 32 the decode keeps in registers), 3 anchors."""
    anch = ANCH[:3]
    rng = np.random.default_rng(40)
    maps = rng.normal(0, 2, (2, 3 * (5 + 40), 11, 11)).astype(np.float32)
    maps[:, 4::45] += 3.0                                 # confident objectness
    cnt, det = _run_maps(maps, 0.02, 0.45, 4096, anch, 40)
    for f in range(2):
        n, ref_n, nd = _check_frame(maps[f].astype(np.float64), int(cnt[f]), det[f], 0.02, 0.45, 4096, anch, 40)
        print("frame %d: %d kept (oracle %d), %d near-threshold differences" % (f, n, ref_n, nd))
        assert n > 10


def test_detect_truncation_and_empty():
    rng = np.random.default_rng(5)
    maps = rng.normal(0, 2, (2, len(ANCH) * (5 + C), 13, 13)).astype(np.float32)
    cnt, det = _run_maps(maps, 0.02, 0.45, 3)           # more kept boxes than rows
    for f in range(2):
        ref_n, ref = region.detect(maps[f:f + 1].astype(np.float64), ANCH, C, 0.02, 0.45, 3)[0]
        assert cnt[f] > 3 and abs(int(cnt[f]) - ref_n) <= 2
        _check_frame(maps[f].astype(np.float64), int(cnt[f]), det[f], 0.02, 0.45, 3)
    cnt, _ = _run_maps(maps, 1.0, 0.45, 8)               # no score exceeds 1
    assert (cnt == 0).all()


def test_region_argument_errors():
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.NetSpec("head", 8, [synth.Layer(1, 125, False, synth.ACT_LINEAR, synth.POOL_NONE)])
    with make_net(spec, prec="fp32", max_batch=2, max_side=13) as net:
        d = torch.zeros(16, device="cuda")
        with pytest.raises(binding.NetError) as e:
            net.detect_device(d, 1, 13, 13, d, d)
        assert e.value.status == binding.NET_E_STATE
        with pytest.raises(binding.NetError) as e:
            net.set_region(ANCH, 19, 0.1, 0.45, 10)      # 5 x (5 + 19) != 125
        assert e.value.status == binding.NET_E_INVAL
        net.set_region(ANCH, C, 0.1, 0.45, 10)
        with pytest.raises(binding.NetError) as e:
            net.detect_device(d, 3, 13, 13, d, d)        # batch beyond max_batch
        assert e.value.status == binding.NET_E_SHAPE
        with pytest.raises(binding.NetError) as e:
            net.detect_device(d, 1, 14, 13, d, d)        # grid beyond max_side's
        assert e.value.status == binding.NET_E_SHAPE
    big = synth.NetSpec("head", 8, [synth.Layer(1, 125, False, synth.ACT_LINEAR, synth.POOL_NONE)])
    with make_net(big, prec="fp32", max_batch=1, max_side=32) as net:   # 32 x 32 x 5 boxes > 4096
        with pytest.raises(binding.NetError) as e:
            net.set_region(ANCH, C, 0.1, 0.45, 10)
        assert e.value.status == binding.NET_E_UNSUPPORTED


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_forward_detect_9conv_416(prec):
    """The 9-conv network's 125-channel 13 x 13 map decoded on the device.
    Frames -> detections through one call equals the device forward pass
    followed by net_detect_device bit for bit; the detections are valid for
    the oracle decode of the GPU's own map; against the exact FP64 network
    (FP32 path only, whose map is within 1e-4) the kept sets agree up to
    near-threshold decisions."""
    import torch
    spec = synth.net_9conv()
    _, x, blob = synth.workload_net(spec, synth.SEED_9CONV, 2, 416, 416)
    thr, nms_thr, md = 0.04, 0.45, 512
    with make_net(spec, prec=prec, max_batch=2, max_side=416) as net:
        net.load_weights(blob)
        net.set_region(ANCH, C, thr, nms_thr, md)
        cnt, det = net.forward_detect(x)
        d_x = torch.from_numpy(x).cuda()
        d_map = torch.empty((2, 125, 13, 13), device="cuda")
        net.forward_device(d_x, 2, 416, 416, d_map)
        d_cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
        d_det = torch.zeros(2 * md * 32, dtype=torch.uint8, device="cuda")
        net.detect_device(d_map, 2, 13, 13, d_cnt, d_det)
        torch.cuda.synchronize()
        from paper_1811_03882_gb300.binding import DETECTION
        det2 = d_det.cpu().numpy().view(DETECTION).reshape(2, md)
        gmap = d_map.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(cnt, d_cnt.cpu().numpy())
    for f in range(2):
        np.testing.assert_array_equal(det[f][:cnt[f]], det2[f][:cnt[f]])
        n, ref_n, nd = _check_frame(gmap[f], int(cnt[f]), det[f], thr, nms_thr, md)
        print("%s frame %d: %d kept, oracle on the GPU's map %d, %d near-threshold differences" %
              (prec, f, n, ref_n, nd))
        assert n > 0
    if prec == "fp32":
        ex = oracle.forward(spec.layers, 3, x, blob)
        assert oracle.normwise_rel_err(gmap, ex) <= 1e-4
        for f in range(2):
            ref_n, ref = region.detect(ex[f:f + 1], ANCH, C, thr, nms_thr, md)[0]
            got = {(int(d["cls"]), int(d["id"])) for d in det[f][:cnt[f]]}
            assert len(got ^ {(r[0], r[1]) for r in ref}) <= max(2, ref_n // 50)
