// tune.cu — genetic search over per-layer operand precision.
//
// The paper's offload search (Sec. 3.3 and 4; parameters in Sec. 5.1.2)
// encodes one bit per parallelisable loop (1 = run it on the GPU), measures
// each candidate program, scores it with fitness = (time)^(-1/2), keeps the
// best individual unchanged (elitism), picks parents by roulette in
// proportion to fitness, crosses them at one point with rate Pc = 0.9,
// flips each bit with rate Pm = 0.05, reuses the measurement of a gene seen
// before instead of re-running it, and scores a run that exceeds the time
// limit as if it took 1000 s.  Here the same search runs over the choice
// the paper's loops have no counterpart for but this pass does: one bit per
// FP8-capable layer, 1 = E4M3 operands, 0 = BF16.  A plan whose output
// leaves the error budget (normwise max relative error against the FP32
// path on the caller's frames) is scored like the paper's timed-out runs.
// Times are CUDA-event measurements of the whole forward pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/net.h"
#include "common.cuh"
#include "kernels.h"
#include "net_internal.h"

using namespace dn;

namespace {

struct Rng {   // SplitMix64 stream
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    int below(int n) { return (int)(next() % (uint64_t)n); }
};

struct Eval {
    double ms = 0.0, err = 0.0, fitness = 0.0;
};

constexpr double kTimeoutMs = 1.0e6;   // the paper's "counts as 1000 s"

// The paper's GA over integer genes, gene i taking values in [0, alpha[i])
// (two-valued genes are the paper's bits).  evaluate(gene) returns its Eval
// (memoised by the caller).  The first individual is `seed`; the best
// individual ever seen is returned in best / best_g.
template <class Evaluate>
void ga_run(const std::vector<int>& alpha, const net_ga_opts* opt, const std::vector<int>& seed, Evaluate evaluate,
            std::vector<int>* best_g, Eval* best) {
    const int a = (int)alpha.size();
    Rng rng{opt->seed ? opt->seed : 0x1811038820ull};
    std::vector<std::vector<int>> pop(opt->population, std::vector<int>(a));
    for (auto& g : pop)
        for (int i = 0; i < a; ++i) g[i] = rng.below(alpha[i]);
    pop[0] = seed;
    *best_g = seed;
    best->fitness = -1.0;
    for (int gen = 0; gen < opt->generations; ++gen) {
        std::vector<Eval> ev(pop.size());
        double fsum = 0.0;
        int elite = 0;
        for (size_t i = 0; i < pop.size(); ++i) {
            ev[i] = evaluate(pop[i]);
            fsum += ev[i].fitness;
            if (ev[i].fitness > ev[elite].fitness) elite = (int)i;
            if (ev[i].fitness > best->fitness) {
                *best = ev[i];
                *best_g = pop[i];
            }
        }
        if (gen + 1 == opt->generations) break;
        // next generation: elite kept unchanged, the rest bred from roulette parents
        auto roulette = [&]() -> const std::vector<int>& {
            double r = rng.uniform() * fsum;
            for (size_t i = 0; i < pop.size(); ++i) {
                r -= ev[i].fitness;
                if (r <= 0) return pop[i];
            }
            return pop.back();
        };
        std::vector<std::vector<int>> next;
        next.push_back(pop[elite]);
        while ((int)next.size() < opt->population) {
            std::vector<int> p1 = roulette(), p2 = roulette();
            if (a > 1 && rng.uniform() < opt->crossover) {
                const int cut = 1 + rng.below(a - 1);
                for (int i = cut; i < a; ++i) std::swap(p1[i], p2[i]);
            }
            for (auto* ch : {&p1, &p2}) {
                // mutation: a bit flips; a many-valued gene takes another value
                for (int i = 0; i < a; ++i)
                    if (rng.uniform() < opt->mutation && alpha[i] > 1)
                        (*ch)[i] = alpha[i] == 2 ? (*ch)[i] ^ 1 : ((*ch)[i] + 1 + rng.below(alpha[i] - 1)) % alpha[i];
                if ((int)next.size() < opt->population) next.push_back(*ch);
            }
        }
        pop.swap(next);
    }
}

}  // namespace

extern "C" net_status net_tune_precision(net_t* n, const float* d_frames, int batch, int h, int w,
                                         const net_ga_opts* opt, int* prec_out, net_ga_result* res) {
    if (!n || !d_frames || !opt || !prec_out || !res) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    if (opt->population < 2 || opt->generations < 1 || opt->reps < 1 || !(opt->max_err > 0) ||
        opt->crossover < 0 || opt->crossover > 1 || opt->mutation < 0 || opt->mutation > 1)
        return fail(NET_E_INVAL, "bad search options");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    std::vector<int> genes;   // layer index of each gene
    for (int l = 0; l < (int)n->L.size(); ++l)
        if (n->L[l].fp8_capable) genes.push_back(l);
    if (genes.empty()) return fail(NET_E_STATE, "no FP8-capable layer: create the handle with NET_FP8");
    cudaError_t e = cudaSetDevice(n->device);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "%s", cudaGetErrorString(e));
    const int nl = (int)n->L.size();
    int c, ho, wo;
    net_output_shape(n, h, w, &c, &ho, &wo);
    const size_t nout = (size_t)batch * c * ho * wo;
    float *d_ref = nullptr, *d_out = nullptr;
    if (dn::dalloc(&d_ref, nout * sizeof(float)) != cudaSuccess || dn::dalloc(&d_out, nout * sizeof(float)) != cudaSuccess) {
        dn::dfree(d_ref);
        return fail(NET_E_OOM, "search buffers");
    }
    std::vector<float> ref(nout), out(nout);
    std::vector<int> saved(nl);
    for (int l = 0; l < nl; ++l) saved[l] = n->L[l].prec;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);

    // reference: the FP32 path over the same frames
    s = run_fp32_reference(n, d_frames, batch, h, w, d_ref, nullptr);
    // the handle's stream may be non-blocking: finish it before a plain copy
    if (s == NET_OK && (cudaStreamSynchronize(n->stream) != cudaSuccess ||
                        cudaMemcpy(ref.data(), d_ref, nout * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess))
        s = fail(NET_E_CUDA, "reference copy");
    double rmax = 0.0;
    for (float v : ref) rmax = std::max(rmax, (double)std::fabs(v));
    if (rmax == 0.0) rmax = 1.0;

    std::map<std::vector<int>, Eval> memo;
    int evaluations = 0, hits = 0;
    auto evaluate = [&](const std::vector<int>& g) -> Eval {
        auto it = memo.find(g);
        if (it != memo.end()) {
            ++hits;
            return it->second;
        }
        Eval ev;
        for (size_t i = 0; i < genes.size(); ++i) set_layer_format(n->L[genes[i]], g[i] ? NET_FP8 : NET_BF16);
        invalidate_plans(n);
        net_status st = run_forward(n, d_frames, batch, h, w, d_out);   // plans, capture, warm-up
        if (st == NET_OK) {
            cudaEventRecord(e0, n->stream);
            for (int r = 0; r < opt->reps && st == NET_OK; ++r) st = run_forward(n, d_frames, batch, h, w, d_out);
            cudaEventRecord(e1, n->stream);
        }
        float ms = 0.f;
        if (st == NET_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaMemcpy(out.data(), d_out, nout * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
            check_device_error(n) == NET_OK) {
            double d = 0.0;
            for (size_t i = 0; i < nout; ++i) d = std::max(d, std::fabs((double)out[i] - (double)ref[i]));
            ev.ms = ms / opt->reps;
            ev.err = d / rmax;
            if (!std::isfinite(ev.err)) ev.err = 1e30;
        } else {
            ev.ms = kTimeoutMs;
            ev.err = 1e30;
        }
        const double t = ev.err <= opt->max_err ? ev.ms : kTimeoutMs;
        ev.fitness = 1.0 / std::sqrt(t);
        memo[g] = ev;
        ++evaluations;
        return ev;
    };

    const int a = (int)genes.size();
    // One individual starts as the all-BF16 plan, the counterpart of the
    // paper's all-zero gene (everything on the CPU, its reference run): the
    // search then always holds a plan inside the error budget.
    std::vector<int> best_g(a, 0);
    Eval best;
    best.fitness = -1.0;
    if (s == NET_OK) ga_run(std::vector<int>(a, 2), opt, std::vector<int>(a, 0), evaluate, &best_g, &best);
    // reference points for the report
    Eval all_bf16, all_fp8;
    if (s == NET_OK) {
        all_bf16 = evaluate(std::vector<int>(a, 0));
        all_fp8 = evaluate(std::vector<int>(a, 1));
    }
    // leave the handle on the best feasible plan (else on its original formats)
    const bool feasible = best.fitness > 1.0 / std::sqrt(kTimeoutMs) + 1e-12 && best.err <= opt->max_err;
    for (int l = 0; l < nl; ++l) set_layer_format(n->L[l], saved[l]);
    if (feasible)
        for (size_t i = 0; i < genes.size(); ++i) set_layer_format(n->L[genes[i]], best_g[i] ? NET_FP8 : NET_BF16);
    invalidate_plans(n);
    for (int l = 0; l < nl; ++l) prec_out[l] = n->L[l].prec;
    std::memset(res, 0, sizeof(*res));
    res->ms = best.ms;
    res->err = best.err;
    res->ms_all_bf16 = all_bf16.ms;
    res->err_all_bf16 = all_bf16.err;
    res->ms_all_fp8 = all_fp8.ms;
    res->err_all_fp8 = all_fp8.err;
    res->evaluations = evaluations;
    res->memo_hits = hits;
    res->fp8_layers = feasible ? (int)std::count(best_g.begin(), best_g.end(), 1) : -1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dn::dfree(d_ref);
    dn::dfree(d_out);
    if (s != NET_OK) return s;
    if (!feasible) return fail(NET_E_STATE, "no plan within the error budget %g", opt->max_err);
    return NET_OK;
}

// Genetic search over the fixed-batch tile plan: one gene per tensor-core
// layer with more than one valid (N tile, split-K) pair, the same GA as the
// precision search.  Every plan computes the same sums in another order, so
// the error check against the analytic plan's output only guards against a
// broken configuration.
extern "C" net_status net_tune_tiles(net_t* n, const float* d_frames, int batch, int h, int w,
                                     const net_ga_opts* opt, int* bn_out, int* ks_out, net_tile_result* res) {
    if (!n || !d_frames || !opt || !bn_out || !ks_out || !res) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    if (opt->population < 2 || opt->generations < 1 || opt->reps < 1 || !(opt->max_err > 0) ||
        opt->crossover < 0 || opt->crossover > 1 || opt->mutation < 0 || opt->mutation > 1)
        return fail(NET_E_INVAL, "bad search options");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    cudaError_t e = cudaSetDevice(n->device);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "%s", cudaGetErrorString(e));
    const int nl = (int)n->L.size();
    std::vector<int> saved_bn(nl), saved_ks(nl), saved_mb(nl);
    for (int l = 0; l < nl; ++l) {
        saved_bn[l] = n->L[l].tile_bn;
        saved_ks[l] = n->L[l].tile_ks;
        saved_mb[l] = n->L[l].tile_mb;
        n->L[l].tile_bn = n->L[l].tile_ks = n->L[l].tile_mb = 0;   // the analytic plan first
    }
    invalidate_plans(n);
    std::vector<int> genes;                     // layer of each gene
    std::vector<std::vector<TileOpt>> options;  // its (bn, ksplit, CTAs per SM) alphabet
    for (int l = 0; l < nl; ++l) {
        std::vector<TileOpt> o;
        tc_tile_options(n, l, &o);
        if (o.size() > 1) {
            genes.push_back(l);
            options.push_back(o);
        }
    }
    int c, ho, wo;
    net_output_shape(n, h, w, &c, &ho, &wo);
    const size_t nout = (size_t)batch * c * ho * wo;
    float *d_ref = nullptr, *d_out = nullptr;
    if (dn::dalloc(&d_ref, nout * sizeof(float)) != cudaSuccess || dn::dalloc(&d_out, nout * sizeof(float)) != cudaSuccess) {
        dn::dfree(d_ref);
        for (int l = 0; l < nl; ++l) {
            n->L[l].tile_bn = saved_bn[l];
            n->L[l].tile_ks = saved_ks[l];
            n->L[l].tile_mb = saved_mb[l];
        }
        return fail(NET_E_OOM, "search buffers");
    }
    std::vector<float> ref(nout), out(nout);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the analytic plan: its output is the reference, its genes the seed
    std::vector<int> seed(genes.size(), 0);
    Plan* P = nullptr;
    s = get_plan(n, batch, h, w, &P);
    if (s == NET_OK)
        for (size_t i = 0; i < genes.size(); ++i)
            for (size_t j = 0; j < options[i].size(); ++j)
                if (options[i][j].bn == P->runs[genes[i]].BN && options[i][j].ks == P->runs[genes[i]].ksplit &&
                    options[i][j].mb == P->runs[genes[i]].mb)
                    seed[i] = (int)j;
    if (s == NET_OK) s = run_forward(n, d_frames, batch, h, w, d_ref);
    // the handle's stream may be non-blocking: finish it before a plain copy
    if (s == NET_OK && (cudaStreamSynchronize(n->stream) != cudaSuccess ||
                        cudaMemcpy(ref.data(), d_ref, nout * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess))
        s = fail(NET_E_CUDA, "reference copy");
    double rmax = 0.0;
    for (float v : ref) rmax = std::max(rmax, (double)std::fabs(v));
    if (rmax == 0.0) rmax = 1.0;

    std::map<std::vector<int>, Eval> memo;
    int evaluations = 0, hits = 0;
    auto apply = [&](const std::vector<int>& g) {
        for (size_t i = 0; i < genes.size(); ++i) {
            n->L[genes[i]].tile_bn = options[i][g[i]].bn;
            n->L[genes[i]].tile_ks = options[i][g[i]].ks;
            n->L[genes[i]].tile_mb = options[i][g[i]].mb;
        }
        invalidate_plans(n);
    };
    auto evaluate = [&](const std::vector<int>& g) -> Eval {
        auto it = memo.find(g);
        if (it != memo.end()) {
            ++hits;
            return it->second;
        }
        Eval ev;
        apply(g);
        net_status st = run_forward(n, d_frames, batch, h, w, d_out);   // plans, capture, warm-up
        if (st == NET_OK) {
            cudaEventRecord(e0, n->stream);
            for (int r = 0; r < opt->reps && st == NET_OK; ++r) st = run_forward(n, d_frames, batch, h, w, d_out);
            cudaEventRecord(e1, n->stream);
        }
        float ms = 0.f;
        if (st == NET_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaMemcpy(out.data(), d_out, nout * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
            check_device_error(n) == NET_OK) {
            double d = 0.0;
            for (size_t i = 0; i < nout; ++i) d = std::max(d, std::fabs((double)out[i] - (double)ref[i]));
            ev.ms = ms / opt->reps;
            ev.err = std::isfinite(d) ? d / rmax : 1e30;
        } else {
            ev.ms = kTimeoutMs;
            ev.err = 1e30;
        }
        ev.fitness = 1.0 / std::sqrt(ev.err <= opt->max_err ? ev.ms : kTimeoutMs);
        static const bool verbose = getenv("NET_TUNE_VERBOSE") != nullptr;   // diagnostics
        if (verbose) {
            fprintf(stderr, "tile plan [");
            for (size_t i = 0; i < genes.size(); ++i)
                fprintf(stderr, " L%d:%d/%d/%d", genes[i], options[i][g[i]].bn, options[i][g[i]].ks,
                        options[i][g[i]].mb);
            fprintf(stderr, " ] status %d (%s) ms %.4f err %.3e\n", (int)st, st == NET_OK ? "" : net_last_error(),
                    ev.ms, ev.err);
        }
        memo[g] = ev;
        ++evaluations;
        return ev;
    };
    std::vector<int> best_g = seed;
    Eval best;
    best.fitness = -1.0;
    Eval analytic;
    if (s == NET_OK) {
        analytic = evaluate(seed);
        if (!genes.empty()) {
            std::vector<int> alpha;
            for (auto& o : options) alpha.push_back((int)o.size());
            ga_run(alpha, opt, seed, evaluate, &best_g, &best);
        } else {
            best = analytic;
        }
    }
    // leave the best plan set (the analytic one when the search failed)
    const bool found = s == NET_OK && best.fitness > 0 && best.err <= opt->max_err;
    if (getenv("NET_TUNE_VERBOSE"))
        fprintf(stderr, "tile search: status %d best ms %.4f err %.3e fitness %.4f analytic ms %.4f err %.3e found %d\n",
                (int)s, best.ms, best.err, best.fitness, analytic.ms, analytic.err, (int)found);
    if (found) {
        apply(best_g);
    } else {
        for (int l = 0; l < nl; ++l) {
            n->L[l].tile_bn = saved_bn[l];
            n->L[l].tile_ks = saved_ks[l];
            n->L[l].tile_mb = saved_mb[l];
        }
        invalidate_plans(n);
    }
    std::memset(res, 0, sizeof(*res));
    res->ms = found ? best.ms : analytic.ms;
    res->ms_analytic = analytic.ms;
    res->evaluations = evaluations;
    res->memo_hits = hits;
    int changed = 0;
    for (size_t i = 0; i < genes.size(); ++i) changed += found && best_g[i] != seed[i];
    res->changed_layers = changed;
    if (s == NET_OK) s = get_plan(n, batch, h, w, &P);
    if (s == NET_OK)
        for (int l = 0; l < nl; ++l) {
            const bool tc = n->L[l].engine == ENG_TC;
            bn_out[l] = tc ? P->runs[l].BN : 0;
            ks_out[l] = tc ? P->runs[l].ksplit : 0;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dn::dfree(d_ref);
    dn::dfree(d_out);
    if (s != NET_OK) return s;
    if (!found) return fail(NET_E_STATE, "no tile plan within the error budget %g", opt->max_err);
    return NET_OK;
}

// The same search over the grouped launches of an uneven batch (and of the
// serving steps, which use the same per-layer choice): one gene per
// tensor-core layer whose alphabet is (N tile, CTAs per SM, ring stage cap)
// triples, the first of them the analytic choice.  Grouped launches never
// split K, and these genes change neither a frame's sums nor their order,
// so every candidate must reproduce the analytic plan's outputs exactly
// (max_err still bounds them); the time is the whole batch's CUDA-graph
// replay.
extern "C" net_status net_tune_uneven(net_t* n, const float* const* d_in, const int* side, int cnt,
                                      float* const* d_out, const net_ga_opts* opt, net_tile_result* res) {
    if (!n || !d_in || !side || !d_out || !opt || !res || cnt < 1) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    if (opt->population < 2 || opt->generations < 1 || opt->reps < 1 || !(opt->max_err > 0) ||
        opt->crossover < 0 || opt->crossover > 1 || opt->mutation < 0 || opt->mutation > 1)
        return fail(NET_E_INVAL, "bad search options");
    for (auto& L : n->L)
        if (L.engine != ENG_TC) return fail(NET_E_UNSUPPORTED, "uneven batches have grouped launches on tensor cores only");
    for (int f = 0; f < cnt; ++f) {
        net_status s = check_shape(n, 1, side[f], side[f]);
        if (s != NET_OK) return s;
    }
    cudaError_t e = cudaSetDevice(n->device);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "%s", cudaGetErrorString(e));
    const int nl = (int)n->L.size();
    struct Saved {
        int bn, mb, nst;
    };
    std::vector<Saved> saved(nl);
    for (int l = 0; l < nl; ++l) {
        saved[l] = {n->L[l].grp_bn, n->L[l].grp_mb, n->L[l].grp_nst};
        n->L[l].grp_bn = n->L[l].grp_mb = n->L[l].grp_nst = 0;
    }
    auto restore = [&] {
        for (int l = 0; l < nl; ++l) {
            n->L[l].grp_bn = saved[l].bn;
            n->L[l].grp_mb = saved[l].mb;
            n->L[l].grp_nst = saved[l].nst;
        }
        uneven_plans_clear(n);
    };
    uneven_plans_clear(n);
    struct Opt {
        int bn, mb, nst;
    };
    std::vector<int> genes;
    std::vector<std::vector<Opt>> options;
    for (int l = 0; l < nl; ++l) {
        const Layer& L = n->L[l];
        const bool last = l + 1 == nl;
        const int ncols = std::max(L.d.cout, last ? L.d.cout : n->L[l + 1].in_cs);
        std::vector<Opt> o{{0, 1, 0}};   // the analytic choice first
        for (int bn : {0, 64, 128, 256}) {
            if (bn > rup(ncols, 64)) continue;
            if (bn && L.pair && bn < ncols) continue;
            for (int mb = 1; mb <= 2; ++mb) {
                if (mb == 2 && (bn == 0 || bn > 128)) continue;
                for (int nst : {0, 8, 4})
                    if (bn || mb != 1 || nst) o.push_back({bn, mb, nst});
            }
        }
        if (o.size() > 1) {
            genes.push_back(l);
            options.push_back(o);
        }
    }
    // outputs of every frame, concatenated
    std::vector<size_t> nout(cnt);
    size_t total = 0;
    for (int f = 0; f < cnt; ++f) {
        int c, ho, wo;
        net_output_shape(n, side[f], side[f], &c, &ho, &wo);
        nout[f] = (size_t)c * ho * wo;
        total += nout[f];
    }
    std::vector<float> ref(total), out(total);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto gather = [&](std::vector<float>& dst) {
        if (cudaStreamSynchronize(n->stream) != cudaSuccess) return false;
        size_t o = 0;
        for (int f = 0; f < cnt; ++f) {
            if (cudaMemcpy(dst.data() + o, d_out[f], nout[f] * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
                return false;
            o += nout[f];
        }
        return true;
    };
    net_status s = enqueue_uneven(n, d_in, side, cnt, d_out);
    if (s == NET_OK && !gather(ref)) s = fail(NET_E_CUDA, "reference copy");
    if (s == NET_OK) s = check_device_error(n);
    double rmax = 0.0;
    for (float v : ref) rmax = std::max(rmax, (double)std::fabs(v));
    if (rmax == 0.0) rmax = 1.0;
    std::map<std::vector<int>, Eval> memo;
    int evaluations = 0, hits = 0;
    auto apply = [&](const std::vector<int>& g) {
        for (size_t i = 0; i < genes.size(); ++i) {
            Layer& L = n->L[genes[i]];
            L.grp_bn = options[i][g[i]].bn;
            L.grp_mb = options[i][g[i]].mb;
            L.grp_nst = options[i][g[i]].nst;
        }
        uneven_plans_clear(n);
    };
    auto evaluate = [&](const std::vector<int>& g) -> Eval {
        auto it = memo.find(g);
        if (it != memo.end()) {
            ++hits;
            return it->second;
        }
        Eval ev;
        apply(g);
        net_status st = enqueue_uneven(n, d_in, side, cnt, d_out);   // plan, capture, warm-up
        if (st == NET_OK) {
            cudaEventRecord(e0, n->stream);
            for (int r = 0; r < opt->reps && st == NET_OK; ++r) st = enqueue_uneven(n, d_in, side, cnt, d_out);
            cudaEventRecord(e1, n->stream);
        }
        float ms = 0.f;
        if (st == NET_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            gather(out) && check_device_error(n) == NET_OK) {
            double d = 0.0;
            for (size_t i = 0; i < total; ++i) d = std::max(d, std::fabs((double)out[i] - (double)ref[i]));
            ev.ms = ms / opt->reps;
            ev.err = std::isfinite(d) ? d / rmax : 1e30;
        } else {
            ev.ms = kTimeoutMs;
            ev.err = 1e30;
        }
        ev.fitness = 1.0 / std::sqrt(ev.err <= opt->max_err ? ev.ms : kTimeoutMs);
        memo[g] = ev;
        ++evaluations;
        return ev;
    };
    std::vector<int> seed(genes.size(), 0), best_g = seed;
    Eval best, analytic;
    best.fitness = -1.0;
    if (s == NET_OK) {
        analytic = evaluate(seed);
        if (!genes.empty()) {
            std::vector<int> alpha;
            for (auto& o : options) alpha.push_back((int)o.size());
            ga_run(alpha, opt, seed, evaluate, &best_g, &best);
        } else {
            best = analytic;
        }
    }
    const bool found = s == NET_OK && best.fitness > 0 && best.err <= opt->max_err;
    if (found) apply(best_g);
    else restore();
    std::memset(res, 0, sizeof(*res));
    res->ms = found ? best.ms : analytic.ms;
    res->ms_analytic = analytic.ms;
    res->evaluations = evaluations;
    res->memo_hits = hits;
    int changed = 0;
    for (size_t i = 0; i < genes.size(); ++i) changed += found && best_g[i] != seed[i];
    res->changed_layers = changed;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != NET_OK) return s;
    if (!found) return fail(NET_E_STATE, "no grouped plan within the error budget %g", opt->max_err);
    return NET_OK;
}

extern "C" net_status net_plan_grouped(const net_t* n, int* bn, int* mb, int* nst, int cnt) {
    if (!n || !bn || !mb || !nst) return fail(NET_E_INVAL, "NULL argument");
    if (cnt < (int)n->L.size()) return fail(NET_E_INVAL, "need %d entries", (int)n->L.size());
    for (size_t l = 0; l < n->L.size(); ++l) {
        bn[l] = n->L[l].grp_bn;
        mb[l] = n->L[l].grp_mb;
        nst[l] = n->L[l].grp_nst;
    }
    return NET_OK;
}
