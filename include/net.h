/*
 * net.h — C ABI of the device-resident CNN forward-pass library (sm_103a).
 *
 * The paper (Yamato et al., Sec. 3.2) reduces CPU<->GPU traffic by hoisting
 * every copy of a GPU loop's data to the outermost loop that does not touch
 * it on the CPU, so that data moves once instead of once per loop.  This
 * library takes that rule to its limit for the loop nests that dominate the
 * Darknet workload the paper offloads (Sec. 5.1.1): the convolutional
 * network forward pass.  Weights are uploaded once (net_load_weights); a
 * frame crosses host->device once and its result device->host once
 * (net_forward); every activation in between stays in device memory.
 *
 * Layer semantics (conv stride 1, pad k/2; batchnorm folded into the
 * weights; bias; leaky rectifier 0.1 or linear; optional 2x2 max pool) are
 * the plain definitions of a Darknet convolutional layer; the paper prints
 * none of them.
 *
 * Conventions for every entry point:
 *  - Host buffers are owned by the caller and only read/written during the
 *    call (net_submit copies the frame before returning).
 *  - Device pointers ("d_" prefix) are CUDA device addresses on the
 *    handle's device, owned by the caller, used in stream order on the
 *    handle's stream.
 *  - Frames are NCHW float32, C = in_c; results are NCHW float32 with the
 *    last layer's channel count and the spatial size after all pools.
 *  - Every call returns a net_status; nothing aborts.  The message of the
 *    last failure on the calling thread is available from net_last_error.
 *  - A handle is not safe for concurrent net_forward* calls; the request
 *    queue entry points (net_submit .. net_stats) are thread-safe.
 */
#ifndef NET_H_
#define NET_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct net net_t;

typedef enum {
    NET_OK = 0,
    NET_E_INVAL = 1,       /* bad argument (NULL, size, capacity)            */
    NET_E_SHAPE = 2,       /* frame shape outside what the handle supports   */
    NET_E_WEIGHTS = 3,     /* blob length mismatch / weights not loaded      */
    NET_E_OOM = 4,         /* device allocation failed                       */
    NET_E_BUDGET = 5,      /* request needs more than the HBM budget         */
    NET_E_TIMEOUT = 6,     /* net_wait timed out                             */
    NET_E_CUDA = 7,        /* a CUDA call failed (message kept)              */
    NET_E_DEVICE_WAIT = 8, /* a bounded device-side wait gave up             */
    NET_E_STATE = 9,       /* call not valid in the handle's current state   */
    NET_E_UNSUPPORTED = 10 /* configuration not built into this library      */
} net_status;

typedef enum { NET_FP32 = 0, NET_BF16 = 1, NET_FP8 = 2 } net_precision;
typedef enum { NET_ACT_LINEAR = 0, NET_ACT_LEAKY = 1 } net_act;
typedef enum { NET_POOL_NONE = 0, NET_POOL_2X2S2 = 1, NET_POOL_2X2S1_SAME = 2 } net_pool;

/* One convolutional layer: k in {1,3}, stride 1, zero pad k/2.
 * bn != 0: batchnorm (running statistics) folded into W and bias;
 * act: NET_ACT_*; pool: NET_POOL_* (2x2 stride 2 needs even H, W; the
 * stride-1 "same" pool keeps the size, its window clipped at bottom/right). */
typedef struct {
    int k, cout, bn, act, pool;
} net_layer;

typedef struct {
    int in_c;                 /* frame channels                                  */
    int n_layers;
    const net_layer* layers;  /* copied by net_create                            */
    int prec;                 /* net_precision of the conv operands (bulk)       */
    const int* layer_prec;    /* optional per-layer net_precision, or NULL       */
    int max_batch;            /* largest batch for net_forward*                  */
    int max_side;             /* largest frame height/width                      */
    size_t hbm_budget_bytes;  /* activation budget of the request queue; 0: 40 GB */
    void* cuda_stream;        /* cudaStream_t for all work; NULL: an own stream that
                                 synchronises with the legacy default stream  */
    int device;               /* CUDA device ordinal                             */
} net_desc;

/* Creates a handle: validates the layer list, plans the device activation
 * arena for (max_batch, max_side) and allocates it.  *out is set on NET_OK.
 * Paper Sec. 3.2: the device buffers of the offloaded loops are created once,
 * outside them, so that no pass allocates or copies per layer. */
net_status net_create(const net_desc* desc, net_t** out);

/* Paper Sec. 3.2 (data a GPU loop only reads crosses to the device once,
 * before the outermost loop): the weights.
 * Uploads the float32 weight blob (host, caller-owned, copied once) and
 * folds it on the device in FP64: s = gamma/sqrt(var+1e-5), W' = W*s,
 * b' = beta - mean*s, then reorders W' to [cout][kh][kw][cin] and casts it
 * to each layer's precision (FP8: per-output-channel scale max|W'_o|/448).
 * Blob layout per layer: [beta, gamma, mean, var] (cout each) if bn, else
 * [bias] (cout); then W as [cout][cin][k][k].  n_floats must equal the
 * layers' total, else NET_E_WEIGHTS. */
net_status net_load_weights(net_t* net, const float* blob, size_t n_floats);

/* FP8 layers: static per-tensor scale of each layer's input activation
 * (value = code * scale).  scales has n = n_layers entries (host), each
 * positive and finite (else NET_E_INVAL).  The paper runs in one precision;
 * the scales belong to this library's FP8 format. */
net_status net_set_act_scales(net_t* net, const float* scales, int n);

/* No paper counterpart (FP8 format of this library).
 * Measures FP8 activation scales on the device: runs the FP32 copy of the
 * folded weights over the caller's frames (device NCHW float32) and sets
 * scale_l = max|input of layer l| / 448.  Writes them to scales_out (host,
 * n_layers floats) when it is not NULL. */
net_status net_calibrate(net_t* net, const float* d_frames, int batch, int h, int w,
                         float* scales_out);

/* Output shape of the network for an h x w frame. */
net_status net_output_shape(const net_t* net, int h, int w, int* c, int* ho, int* wo);

/* Paper Sec. 3.2 (copies hoisted to the outermost loop) and Sec. 5.1.1 (the
 * Darknet image-analysis pass that is offloaded): synchronous forward pass
 * from host memory: one host->device copy of the batch, the whole network on
 * the device, one device->host copy of the result.  in_nchw: batch x in_c x
 * h x w float32 (host, caller-owned); out_cap_floats must hold
 * batch*c*ho*wo floats (else NET_E_INVAL); NET_E_SHAPE for a batch or side
 * beyond the handle's maxima or an odd size before a 2x2/s2 pool;
 * NET_E_DEVICE_WAIT when a bounded device-side wait expired. */
net_status net_forward(net_t* net, const float* in_nchw, int batch, int h, int w,
                       float* out_nchw, size_t out_cap_floats);

/* Paper Sec. 3.2, as net_forward.
 * Asynchronous form of net_forward for a stream of batches: enqueues the
 * host->device copy of in_nchw (on an upload stream), the forward pass (on
 * the handle's stream) and the device->host copy into out_nchw (on a
 * download stream), and returns.  Two device staging slots alternate, so
 * the copies of one call overlap the pass of the previous one; before a
 * slot is reused the call waits until that slot's previous work finished.
 * The caller keeps in_nchw unchanged and out_nchw unread until
 * net_forward_wait returns (host buffers should be pinned: pageable copies
 * serialise).  Arguments and errors as net_forward. */
net_status net_forward_async(net_t* net, const float* in_nchw, int batch, int h, int w,
                             float* out_nchw, size_t out_cap_floats);

/* Blocks until every net_forward_async call of the handle has finished;
 * returns the first error of the batch of calls (NET_E_DEVICE_WAIT when a
 * bounded device-side wait expired). */
net_status net_forward_wait(net_t* net);

/* Paper Sec. 3.2: the pass with its data already on the device.
 * Stream-ordered forward pass between device buffers (no host copies, no
 * synchronisation).  d_in: batch x in_c x h x w float32, d_out: batch x c x
 * ho x wo float32, both device memory owned by the caller; errors as
 * net_forward (a device-wait expiry shows on a later call). */
net_status net_forward_device(net_t* net, const float* d_in, int batch, int h, int w,
                              float* d_out);

/* As net_forward_device, and also writes every layer's output (after its
 * pool) as NCHW float32 into d_layer_out[l] (device pointers, one per
 * layer, each sized for that layer's output): the values the next layer
 * reads, FP8 codes times their scale.  Diagnostic path (per-layer error
 * against the oracle); the paper has no counterpart. */
net_status net_forward_trace(net_t* net, const float* d_in, int batch, int h, int w,
                             float* const* d_layer_out);

/* Paper Sec. 1 and 5.1.1 (frames from many shared cameras analysed by one
 * service) with the transfer rule of Sec. 3.2.
 * Uneven batch: n frames of different square sides in one pass.  Frame i
 * is d_in[i] (1 x in_c x side[i] x side[i], device) and its result goes to
 * d_out[i].  Every layer of every frame runs in one grouped launch per
 * layer (frames share no reduction, so each result equals the frame's own
 * net_forward_device result bit for bit).  Stream-ordered. */
net_status net_forward_uneven(net_t* net, const float* const* d_in, const int* side, int n,
                              float* const* d_out);

/* ---- detection post-processing -----------------------------------------
 * Paper Sec. 5.1.1: the offloaded benchmark is Darknet's "detection" app;
 * with the transfer rule of Sec. 3.2 the network's final map is decoded on
 * the device and only the detections cross back.  The map is read as the
 * region output of an anchor-box detector: anchor a owns channels
 * a*(5+C) .. a*(5+C)+4+C (tx, ty, tw, th, objectness logit, C class logits);
 * cell (i, j) and anchor a form box id (i*GW + j)*A + a, centred at
 * ((j + sigmoid(tx))/GW, (i + sigmoid(ty))/GH) with size
 * (exp(tw)*pw/GW, exp(th)*ph/GH) as fractions of the frame; the class-c
 * score is sigmoid(to) * softmax(logits)_c.  Boxes scoring above
 * score_thresh in a class are its candidates; greedy non-maximum
 * suppression per class takes them by score (descending, equal scores by
 * id) and drops a box whose IoU with a kept box of its class exceeds
 * nms_iou.  A frame's detections are its kept boxes class by class
 * (ascending), each class in that order, at most max_det of them; its count
 * is the number kept before that cut.  Decode, then suppression and
 * compaction, run in FP32 in two kernels; the result does not depend on the order in
 * which the device appended candidates. */
#define NET_REGION_MAX_ANCHORS 16
typedef struct {
    int n_anchors;          /* A (1 .. NET_REGION_MAX_ANCHORS)                  */
    int n_classes;          /* C; the last layer must have A * (5 + C) outputs  */
    float anchors[2 * NET_REGION_MAX_ANCHORS]; /* (pw, ph) per anchor, in grid cells */
    float score_thresh;     /* candidate when objectness * p(class) > this      */
    float nms_iou;          /* dropped when IoU with a kept box exceeds this    */
    int max_det;            /* detections reported per frame                    */
} net_region;

typedef struct {
    float x, y, w, h;       /* centre and size, fractions of the frame          */
    float score;            /* objectness * p(class)                            */
    int cls;                /* class                                            */
    int id;                 /* box id (i*GW + j)*A + a                          */
    int pad;
} net_detection;            /* 32 bytes                                         */

/* Sets the decode and suppression parameters (copied) and allocates their
 * device buffers for max_batch frames of the largest grid the handle's
 * max_side gives.  NET_E_INVAL for a parameter out of range or a last layer
 * whose output count is not A * (5 + C); NET_E_UNSUPPORTED when that grid
 * times A exceeds 4096 boxes (the suppression sorts a class's candidates in
 * shared memory). */
net_status net_set_region(net_t* net, const net_region* region);

/* Stream-ordered detection of a device map (batch x A*(5+C) x gh x gw
 * float32, NCHW, caller-owned): d_counts[batch] kept boxes per frame and
 * d_det[batch][max_det] the detections (device memory, caller-owned; rows
 * past a frame's count are left as they were).  NET_E_STATE without
 * net_set_region; NET_E_SHAPE for a batch or grid beyond its set-up. */
net_status net_detect_device(net_t* net, const float* d_map, int batch, int gh, int gw, int* d_counts,
                             net_detection* d_det);

/* Frames (host NCHW float32) to detections: one host->device copy of the
 * batch, the forward pass and the detection on the device, one
 * device->host copy of the counts and detections.  counts: batch ints;
 * det: batch * max_det detections (host, caller-owned). */
net_status net_forward_detect(net_t* net, const float* in_nchw, int batch, int h, int w, int* counts,
                              net_detection* det);

/* ---- nightmare pass (gradient of a layer's energy) -----------------------
 * Paper Sec. 5.1.1: the offloaded benchmark also runs Darknet's "nightmare"
 * app, which changes an image by gradient ascent so that it excites a chosen
 * layer more.  The objective of layer L is J = 1/2 * sum of the squares of
 * its output (after its pool); its gradient with respect to the frames flows
 * back through max pools (to the first maximum of each window, scan order
 * (0,0), (0,1), (1,0), (1,1); the stride-1 pool gathers what the windows a
 * position wins send it), leaky rectifiers (times 1 where the activation is
 * positive, 0.1 elsewhere) and convs (backward-data: a conv with the folded
 * weights transposed and flipped, on the same CUDA-core kernel as the
 * forward pass; the batchnorm scale comes with the folded weights).  It runs
 * on the FP32 path: the handle's every layer NET_FP32 (NET_E_UNSUPPORTED
 * otherwise); the first call allocates its buffers for (max_batch,
 * max_side) and builds the backward weights (rebuilt after
 * net_load_weights). */

/* d_in: batch x in_c x h x w float32 frames, d_grad: the same shape (device,
 * caller-owned): dJ/d(frames) for layer `layer`; objective (host, batch
 * doubles, may be NULL): J per frame.  Returns when done. */
net_status net_nightmare_grad(net_t* net, const float* d_in, int batch, int h, int w, int layer, float* d_grad,
                              double* objective);

/* As net_nightmare_grad, and also writes, for every layer l <= layer, its
 * activation before its pool into d_act[l] (batch x cout x H_l x W_l, the
 * conv's output size) and the gradient with respect to its output (after
 * its pool) into d_gout[l] (NCHW float32, device pointers, one per layer,
 * each sized for that tensor).  Diagnostic path (per-layer checks against
 * the oracle); the paper has no counterpart. */
net_status net_nightmare_trace(net_t* net, const float* d_in, int batch, int h, int w, int layer, float* d_grad,
                               float* const* d_act, float* const* d_gout);

/* One ascent step on device frames in place: x += rate * g / mean(|g|) with
 * g = dJ/dx of each frame over that frame (mean over its in_c*h*w values);
 * objective (host, may be NULL): J per frame before the step. */
net_status net_nightmare_step(net_t* net, float* d_frames, int batch, int h, int w, int layer, float rate,
                              double* objective);

/* ---- Jacobi solver of the Laplace equation ------------------------------
 * Paper Sec. 4: the sample application that solves the Laplace equation by
 * the Jacobi method (13.5x there), run with the transfer rule of Sec. 3.2:
 * the grid crosses to the device once, every sweep stays in device memory,
 * the result crosses back once.  The grid is ny x nx float32, row-major;
 * its first and last rows and columns are fixed boundary values.  A sweep
 * replaces every interior point by the mean of its four neighbours in the
 * previous iterate; the change of a sweep is the largest |new - old| over
 * the interior; sweeps repeat while the last change exceeds tol and fewer
 * than iter_max have run (tol = 0: exactly iter_max sweeps).  The stopping
 * rule is applied on the device; the host polls a 16-byte state once per 16
 * queued sweeps, and sweeps queued past the stop return at once.  FP32. */
typedef struct net_jacobi net_jacobi_t;

/* Handle for one grid size on `device` (work on cuda_stream; NULL: an own
 * stream); allocates two device grids.  NET_E_INVAL unless 3 <= ny, nx <=
 * 65536 (a grid needs an interior). */
net_status net_jacobi_create(int ny, int nx, int device, void* cuda_stream, net_jacobi_t** out);

/* Solves from host grid_in into host grid_out (ny * nx floats each,
 * caller-owned; may be the same buffer); *sweeps and *change (either may be
 * NULL) report the sweeps run and the last change.  NET_E_INVAL for tol < 0
 * or iter_max < 0; iter_max = 0 returns the input. */
net_status net_jacobi_solve(net_jacobi_t* j, const float* grid_in, float tol, int iter_max, float* grid_out,
                            int* sweeps, float* change);

/* As net_jacobi_solve between device grids (caller-owned, row-major ny x
 * nx); returns when done. */
net_status net_jacobi_solve_device(net_jacobi_t* j, const float* d_in, float tol, int iter_max, float* d_out,
                                   int* sweeps, float* change);

/* Kernels the handle has launched (one per queued sweep). */
net_status net_jacobi_launches(const net_jacobi_t* j, uint64_t* total);

/* Releases the handle's device and host memory.  NULL is accepted. */
net_status net_jacobi_free(net_jacobi_t* j);

/* ---- request queue (continuous batching) ------------------------------
 * Paper Sec. 1 and 5.1.1: a camera image-analysis service shared by many
 * cameras and uses.
 * net_submit copies one frame (host NCHW float32, 1 x in_c x h x w) into a
 * pinned staging arena and returns a request id.  A scheduler thread admits
 * queued requests first come, first served while the in-flight cap, the
 * staging arena and the HBM activation budget allow, and runs the requests
 * admitted together as one step: one forward pass of all of them, every
 * layer one grouped launch over the step's frames.  Two steps are in flight
 * at once: requests that arrive while a step runs are admitted into the
 * next one, whose frames upload while the first computes and whose kernels
 * follow the first's on the device; a finished step frees its budget for
 * the requests still queued.  A frame's result does not depend on the other
 * frames of its step.  A frame whose activations exceed the whole budget
 * fails with NET_E_BUDGET; NET_E_SHAPE for a side beyond the handle's
 * maximum. */
net_status net_submit(net_t* net, const float* frame, int h, int w, uint64_t* req_id);

/* Non-blocking: *done = 1 and the result copied to out when finished. */
net_status net_poll(net_t* net, uint64_t req_id, float* out, size_t cap_floats, int* done);

/* Blocks up to timeout_ms (negative: forever); NET_E_TIMEOUT if not done. */
net_status net_wait(net_t* net, uint64_t req_id, float* out, size_t cap_floats, int timeout_ms);

/* Completed-request statistics since the queue started: throughput and
 * latency percentiles (completion minus submission). */
net_status net_stats(net_t* net, double* fps, double* p50_ms, double* p99_ms);

/* Restarts the statistics of net_stats (e.g. after a warm-up period). */
net_status net_stats_reset(net_t* net);

/* ---- per-layer precision ------------------------------------------------
 * A handle created with NET_FP8 keeps, for every tensor-core layer, both an
 * E4M3 and a BF16 copy of its folded weights, so each such layer can run in
 * either format.  net_set_layer_prec takes n_layers net_precision values
 * (other layers must keep the precision they were created with). */
net_status net_set_layer_prec(net_t* net, const int* layer_prec, int n);
net_status net_get_layer_prec(const net_t* net, int* layer_prec, int n);

/* Paper Sec. 3.3 and 4 (the GA), Sec. 5.1.2 (its parameters).
 * Genetic search over the FP8/BF16 choice of every switchable layer: the
 * paper's offload search (Sec. 3.3, 4; parameters of Sec. 5.1.2) with one
 * gene per layer instead of per loop.  Fitness is (time per forward pass in
 * ms)^(-1/2); a plan whose output on d_frames deviates from the FP32 path by
 * more than max_err (normwise max relative error) scores as a 10^6 ms run,
 * like the paper's timed-out individuals; the best individual survives
 * unchanged; parents are drawn by roulette; single-point crossover with
 * probability `crossover`, bit-flip mutation with probability `mutation`;
 * a gene seen before reuses its measurement.  FP8 activation scales must be
 * set (net_calibrate).  On NET_OK the handle is left on the best plan and
 * layer_prec_out (n_layers entries) holds it; NET_E_STATE if no plan met
 * the budget (the handle keeps its previous formats). */
typedef struct {
    int population;          /* M (paper: 30, at most the gene length)        */
    int generations;         /* T (paper: 20)                                 */
    double crossover;        /* Pc (paper: 0.9)                               */
    double mutation;         /* Pm (paper: 0.05)                              */
    double max_err;          /* error budget against the FP32 path            */
    int reps;                /* timed forward passes per evaluation            */
    unsigned long long seed; /* search random stream (0: fixed default)        */
} net_ga_opts;

typedef struct {
    double ms, err;                  /* best plan                               */
    double ms_all_bf16, err_all_bf16;/* every switchable layer in BF16          */
    double ms_all_fp8, err_all_fp8;  /* every switchable layer in FP8           */
    int evaluations, memo_hits, fp8_layers;
} net_ga_result;

net_status net_tune_precision(net_t* net, const float* d_frames, int batch, int h, int w,
                              const net_ga_opts* opts, int* layer_prec_out, net_ga_result* result);

/* No paper counterpart (the tile plan of this library's conv kernel; the
 * search below applies the paper's GA to it).
 * Tile plan of one tensor-core layer for the fixed-batch passes
 * (net_forward*): N tile bn in {64, 128, 256} and split-K factor ksplit in
 * {1, 2, 4, 8, 16}; 0 keeps the analytic choice.  A value the layer cannot take
 * (bn above its padded output columns, ksplit with fewer than four K steps
 * per slice) is NET_E_INVAL.  A BF16 3x3 first layer over at most 8 input
 * channels and at most 256 outputs runs as tap pairs (two taps per MMA over
 * 8-channel pixels) with its weights resident in shared memory: it takes
 * ksplit 1 and an N tile that covers all of its output columns only.
 * Captured graphs and plans are rebuilt. */
net_status net_set_layer_tiles(net_t* net, int layer, int bn, int ksplit);

/* CTAs per SM of one tensor-core layer's fixed-batch launches: 1, 2 (N
 * tiles of at most 128 columns: two CTAs share an SM, each with half the
 * shared memory and at most 80 registers a thread, which doubles the
 * epilogue warps an SM) or 0 (chosen per launch).  NET_E_INVAL otherwise;
 * no paper counterpart (the search below tunes it with the paper's GA). */
net_status net_set_layer_ctas(net_t* net, int layer, int mb);

/* CTAs per SM of every layer's fixed-batch launch for a batch x h x w pass
 * (0 for CUDA-core layers). */
net_status net_plan_ctas(net_t* net, int batch, int h, int w, int* mb, int n);

/* The tile plan the fixed-batch path uses for a batch x h x w pass, after
 * overrides: bn[n] and ksplit[n] per layer (0 for CUDA-core layers). */
net_status net_plan_tiles(net_t* net, int batch, int h, int w, int* bn, int* ksplit, int n);

/* Paper Sec. 3.2 (data stays on the device between the loops that use it),
 * taken one step further: between the layers of a pass, work starts as
 * soon as the rows it reads are written.  dep[n] per layer of a batch x h x
 * w fixed-batch pass: 1 if the layer waits for the previous layer's row
 * bands (each tile for the previous layer's tile rows under its input rows)
 * instead of for the whole previous kernel, else 0.  Plain forward passes
 * (net_forward*, net_forward_detect) use it; passes with per-layer copies
 * out, calibration or NET_TC_FLOW=0 in the environment do not.  NULL
 * arguments or n < n_layers: NET_E_INVAL. */
net_status net_plan_flow(net_t* net, int batch, int h, int w, int* dep, int n);

/* Paper Sec. 3.3 and 4 (the GA) over this library's tile plan.
 * Genetic search over the tile plan: the same algorithm and options as
 * net_tune_precision (max_err bounds the deviation from the analytic plan's
 * output; every plan computes the same sums, only their order differs), one
 * gene per tensor-core layer whose alphabet is that layer's valid (bn,
 * ksplit, CTAs per SM) triples, mutation drawing another triple; the
 * analytic plan is one of the initial individuals.  On NET_OK the handle
 * keeps the best plan as overrides, bn_out / ksplit_out (n_layers entries)
 * hold it and net_plan_ctas reports its CTAs per SM. */
typedef struct {
    double ms, ms_analytic;          /* best plan / the analytic plan           */
    int evaluations, memo_hits, changed_layers;
} net_tile_result;

net_status net_tune_tiles(net_t* net, const float* d_frames, int batch, int h, int w, const net_ga_opts* opts,
                          int* bn_out, int* ksplit_out, net_tile_result* result);

/* Paper Sec. 3.3 and 4 (the GA) over the grouped launches of an uneven
 * batch (net_forward_uneven; the serving steps use the same per-layer
 * choice): one gene per tensor-core layer whose alphabet is (N tile, CTAs
 * per SM, ring stage cap) triples, the analytic choice first; the time is
 * the whole batch of net_forward_uneven(d_in, side, cnt, d_out) (arguments
 * as there).  Grouped launches never split K and the genes change neither
 * a frame's sums nor their order, so every plan must reproduce the analytic
 * outputs (max_err bounds the difference).  On NET_OK the handle keeps the
 * best plan (net_plan_grouped reports it) and result holds the times.
 * NET_E_UNSUPPORTED when a layer runs on CUDA cores. */
net_status net_tune_uneven(net_t* net, const float* const* d_in, const int* side, int cnt, float* const* d_out,
                           const net_ga_opts* opts, net_tile_result* result);

/* The grouped-launch choice per layer: N tile (0: analytic), CTAs per SM
 * (0 or 1: one; 2: two), ring stage cap (0: as many as fit). */
net_status net_plan_grouped(const net_t* net, int* bn, int* mb, int* nst, int n);

/* Paper Sec. 3.3 measures each candidate's run time; this is the per-layer
 * form of that measurement.
 * Per-layer timing: with enable != 0 every later forward pass records a
 * CUDA event pair around each layer's conv kernel (on the handle's stream;
 * CUDA-graph replays record them too).  net_layer_times waits for the most
 * recent pass and writes each layer's conv-kernel time in milliseconds to
 * ms_out (host, n = n_layers entries). */
net_status net_profile(net_t* net, int enable);

/* Phase trace of the tensor-core conv launches (a diagnostic; the paper has
 * no counterpart).  With enable != 0 (which clears the record) every later
 * fixed-batch forward pass makes each CTA of each tensor-core layer write
 * GPU globaltimer stamps (nanoseconds) at ten points: 0 kernel start,
 * 1 prologue done, 2 first producer past the wait for the previous kernel
 * (a layer on the row-band dataflow has none: its producer's start),
 * 3 first K step ready for the first MMA issuer, 4 its last MMA issued,
 * 5 epilogue warp 2 started, 6 epilogue warp 2 done, 7 epilogue warp 6
 * done, 8 closing barrier passed, 9 epilogue warp 2's last accumulator
 * ready (its last tile's MMAs complete; not written by the tap-pair first
 * layer, whose epilogue is its bound); 0 where nothing was written
 * (CUDA-core layers, grids beyond 512 CTAs).  net_trace_read waits for the
 * handle's stream and copies the record, n_layers x 512 x 10 uint64 in that
 * order, to out (host, cap entries at least); NET_E_STATE if tracing was
 * never enabled. */
net_status net_trace(net_t* net, int enable);
net_status net_trace_read(net_t* net, uint64_t* out, size_t cap);
net_status net_layer_times(net_t* net, double* ms_out, int n);

/* Total number of kernels this handle has launched (a CUDA-graph replay
 * counts every kernel node in the graph). */
net_status net_launches(const net_t* net, uint64_t* total);

/* Fault injection for tests of the failure path; the paper has no
 * counterpart.  Every wait inside the tensor-core conv kernel is bounded;
 * when one expires the kernel records the failure in a flag the host reads,
 * drains its copies and MMAs, frees its tensor memory and returns, so the
 * CUDA context stays usable.  After this call the handle's next
 * fixed-batch pass (net_forward*, not captured in a graph) launches
 * tensor-core layer `layer` with a ~1 ms bound on those waits and one of
 * its K steps never loaded, so the wait for it expires: that pass returns
 * NET_E_DEVICE_WAIT (its output is not valid) and later passes are
 * unaffected.  NET_E_INVAL for a layer that does not run on tensor cores. */
net_status net_inject_device_fault(net_t* net, int layer);

/* The same for the row-band dataflow (the paper has no counterpart): the
 * handle's next fixed-batch pass of batch x h x w runs layer `layer`, which
 * must wait on the previous layer's row bands in that pass (net_plan_flow),
 * with a band count that is never reached and a ~1 ms bound on its waits:
 * its producers' wait expires, the layer drains and returns, and the layers
 * after it are released by its finished-warp count, so the pass ends at
 * once with NET_E_DEVICE_WAIT (its output is not valid) and later passes are
 * unaffected.  NET_E_INVAL for a layer that is not on the dataflow. */
net_status net_inject_flow_fault(net_t* net, int layer, int batch, int h, int w);

/* Canary guard regions, a debug aid for out-of-bounds writes; the paper
 * has no counterpart.  With NET_GUARD=1 in the environment when the
 * process first allocates, every device buffer the library allocates
 * (activations, weights, workspaces, staging, detection, nightmare, Jacobi
 * and serving buffers) has 4 KB of 0xA5 bytes directly before and after
 * it.  A buffer's regions are checked when the library frees it (after a
 * device synchronisation); net_guard_check also checks every live buffer
 * and reports all buffers checked so far (freed and live) and how many had
 * a changed region (a write past an end); both 0 when guards are off.  Host
 * memory is untouched; the regions are freed with their buffers. */
net_status net_guard_check(uint64_t* buffers, uint64_t* corrupted);

/* Test hook for net_guard_check: overwrites the first byte after buffer
 * `index` (address order of the live guarded buffers) by a host-side
 * memset, as a one-element overrun would.  NET_E_STATE when guards are
 * off, NET_E_INVAL for an index past the live buffers. */
net_status net_guard_poke(uint64_t index);

/* ---- conv layer without allocation ------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they call (code running while a CUDA
 * graph is captured, real-time loops that allow no allocation after
 * start-up, hosts with a fixed device-memory budget).
 *
 * One FP32 conv layer: y = pool(act(conv(x, weight) + bias)), stride 1,
 * zero pad k/2, computed by the same split-K FP32 kernels as the network
 * path.  d_x: n x cin x h x w float32 NCHW; d_weight: cout x cin x k x k
 * float32 (batchnorm, if any, already folded in); d_bias: cout floats;
 * d_y: n x cout x h' x w' float32 NCHW (h' = h/2 with the 2x2/s2 pool).
 * act: NET_ACT_*; pool: NET_POOL_NONE or NET_POOL_2X2S2.  All pointers are
 * caller-owned device memory on the current device; work is queued on
 * cuda_stream (NULL: legacy default stream) and not synchronised.
 *
 * It calls no cudaMalloc/cudaFree or allocating library routine.  Every
 * intermediate lives in one static device array of
 * NET_NOALLOC_SCRATCH_BYTES that each device loading the library holds
 * until exit; a layer needing more returns NET_E_INVAL before touching the
 * device.  The first call on a device looks the array's address up (with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset re-creates the
 * device's context and moves the array, so the kept address goes stale:
 * a process that resets a device must not call this entry point on that
 * device afterwards.
 * All calls share the array and a call overwrites what the previous one
 * left there, so calls that may overlap on the GPU (different streams,
 * several host threads) race: serialise them. */
#define NET_NOALLOC_SCRATCH_BYTES (32u << 20)
net_status net_conv2d_f32_noalloc(const float* d_x, int n, int cin, int h, int w,
                                  const float* d_weight, const float* d_bias, int cout, int k,
                                  int act, int pool, float* d_y, void* cuda_stream);

/* Releases every device and host resource of the handle (stops the
 * scheduler thread first).  NULL is accepted. */
net_status net_free(net_t* net);

/* Message of the last failure on the calling thread ("" if none). */
const char* net_last_error(void);

/* Library build identification string (static). */
const char* net_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NET_H_ */
