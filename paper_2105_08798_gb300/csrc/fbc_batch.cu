// Batches of plans: many FBC instances of uneven size, each with its own
// right-hand sides, updated by one fixed sequence of launches -- batched
// forward transforms, projections, ONE persistent contraction launch that
// drains a cost-sorted (longest processing time first) tile queue over all
// instances, batched inverse transforms and zero-mean steps -- captured once
// into a CUDA graph and replayed.
//
// The persistent kernel's CTAs take work with atomicAdd on a counter that is
// reset by the graph; no CTA waits for another, so nothing can spin.
//
// Tensor-core batches (TF32, BF16x2, BF16x3) have two launch forms for the
// contraction.  Queue: the k = 0 items run on the double-float tile in the
// persistent CUDA-core launch, each instance's force operand is split into its
// plan's buffer, and the modes k >= 1 of all instances run in one persistent
// tensor-core launch (one CTA per SM) over a queue of items (instance, mode,
// pad tile, rhs group).  Per instance: the graph holds, for each instance, the
// launches of its own apply (k = 0 multi-rhs double-float tile, force split,
// tensor-core grid) -- when every instance fills the GPU by itself, this
// avoids the queue's per-item overhead.  Both give each instance's own bits.
//
// Autotuning: the order of the contraction queue (LPT or the natural
// instance-major order) and, for the CUDA-core forms, the persistent grid
// size (resident CTAs per SM times the SM count, or fewer); for the tensor
// forms the launch form and, for the queue, the rhs group -- right-hand sides
// per CTA, i.e. the N of the tensor-core tile (N = 2 x rhs) -- which trades
// the table gathers (once per group) against the number of items and their
// balance.  Each candidate is timed on the contraction; none changes the
// results.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "fbc_internal.cuh"

namespace {

struct Item {
    int4 w;
    double cost;
};

}  // namespace

struct fbc_batch {
    int n = 0;
    int precision = 0;
    int device = 0;
    std::vector<fbc_plan*> plans;
    std::vector<int> n_rhs;
    std::vector<Item> con_items[2];  // natural order; [0]: k = 0 items of an FP32 batch, [1]: the rest
    std::vector<int4> fwd, proj, inv, zm;
    // tensor-core forms: launch form (0: persistent queue, 1: per-instance launches), rhs per CTA of the queue
    // (one value for the batch, capped per instance), jobs and their items
    int tc_form = 0;
    int rpc = 0;
    std::vector<fbc::TcJob> tc_jobs;
    fbc::TcJob* d_tc_jobs = nullptr;
    size_t smem_tc = 0;
    fbc::LineArgs* d_largs = nullptr;
    fbc::ContractArgs* d_cargs = nullptr;
    int* d_nrhs = nullptr;
    int4* d_fwd = nullptr;
    int4* d_proj = nullptr;
    int4* d_con[2] = {nullptr, nullptr};
    int4* d_inv = nullptr;
    int4* d_zm = nullptr;
    int* d_counter = nullptr;
    size_t smem_con[2] = {0, 0}, smem_line = 0;
    int sm_count = 152, occupancy[2] = {1, 1}, grid[2] = {152, 152};
    int lpt = 1;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double g_alpha = 0.0, g_beta = 0.0;
    uint32_t g_flags = 0;
    bool graph_valid = false;
    double pair_modes = 0.0;
};

namespace {

int bfail(int code, const char* msg) { return fbc::report_error(code, msg); }

int bcuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return fbc::report_error(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, buf);
}

void free_batch(fbc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    void* bufs[] = {b->d_largs, b->d_cargs, b->d_nrhs, b->d_fwd,   b->d_proj,   b->d_con[0],
                    b->d_con[1], b->d_inv,   b->d_zm,   b->d_counter, b->d_tc_jobs};
    for (void* p : bufs)
        if (p) cudaFree(p);
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
    if (*dst) cudaFree(*dst), *dst = nullptr;
    size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

bool tensor(const fbc_batch* b) { return fbc::is_tensor_precision(b->precision); }

// rhs per CTA of instance i for the batch's choice (capped by what its plan's operand buffer holds)
int inst_rpc(const fbc_batch* b, int i) {
    const fbc::Plan& P = b->plans[i]->p;
    int r = std::min(b->rpc, fbc::contract_tc_max_rpc(P));
    while (r > 1 && !fbc::contract_tc_rpc_fits(P, r)) r--;
    return r;
}

// Tensor-core items (instance, k >= 1, pad tile, rhs group) and jobs for the batch's rhs group; the cost of
// an item is its stages (interface tiles) times the rows of its force operand (the tile's N).
void build_tc_items(fbc_batch* b) {
    b->con_items[1].clear();
    b->tc_jobs.resize(b->n);
    b->smem_tc = 0;
    for (int i = 0; i < b->n; i++) {
        const fbc::Plan& P = b->plans[i]->p;
        const int rpc = inst_rpc(b, i), R = b->n_rhs[i], HW = P.H * P.W;
        const int nbuf = fbc::contract_tc_nbuf_smem(b->precision, HW, 2) <= 227 * 1024 ? 2 : 1;
        b->smem_tc = std::max(b->smem_tc, fbc::contract_tc_nbuf_smem(b->precision, HW, nbuf));
        b->tc_jobs[i] = fbc::contract_tc_job(P, R, rpc, nbuf);
        for (int k = 1; k < P.K; k++)
            for (int tA = 0; tA < P.n_ta; tA++)
                for (int g = 0; g < (R + rpc - 1) / rpc; g++) {
                    const int rg = std::min(rpc, R - g * rpc);
                    b->con_items[1].push_back({make_int4(i, k, tA, g), (double)P.n_tb * (16 + ((2 * rg + 15) / 16) * 16)});
                }
    }
}

std::vector<int4> ordered_items(const fbc_batch* b, int phase, bool lpt) {
    std::vector<Item> it = b->con_items[phase];
    if (lpt) std::stable_sort(it.begin(), it.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
    std::vector<int4> out(it.size());
    for (size_t t = 0; t < it.size(); t++) out[t] = it[t].w;
    return out;
}

cudaError_t enqueue_contract(fbc_batch* b, cudaStream_t st);

// Enqueue the whole batched update on `st` (direct launches, no graph).
cudaError_t enqueue(fbc_batch* b, double alpha, double beta, uint32_t flags, cudaStream_t st) {
    cudaError_t e;
    const bool project = flags & FBC_APPLY_PROJECT_NEUTRAL, zmean = flags & FBC_APPLY_ZERO_MEAN_U;
    if ((e = fbc::launch_batch_line(0, b->d_largs, b->d_fwd, (int)b->fwd.size(), b->smem_line, 0, 0, 0, st, fbc::line_fp32(b->precision)))) return e;
    if (project && (e = fbc::launch_batch_line(1, b->d_largs, b->d_proj, (int)b->proj.size(), 0, 0, 0, 0, st, fbc::line_fp32(b->precision)))) return e;
    if ((e = enqueue_contract(b, st))) return e;
    if ((e = fbc::launch_batch_line(2, b->d_largs, b->d_inv, (int)b->inv.size(), b->smem_line, alpha, beta,
                                    zmean ? 1 : 0, st, fbc::line_fp32(b->precision))))
        return e;
    if (zmean && (e = fbc::launch_batch_line(3, b->d_largs, b->d_zm, (int)b->zm.size(), 0, 0, 0, 0, st, fbc::line_fp32(b->precision)))) return e;
    return cudaSuccess;
}

// The contraction of every instance (after the forward transforms, before the inverse ones).
cudaError_t enqueue_contract(fbc_batch* b, cudaStream_t st) {
    cudaError_t e;
    if (tensor(b) && b->tc_form == 1) {
        for (int i = 0; i < b->n; i++)
            if ((e = fbc::launch_contract(b->plans[i]->p, b->n_rhs[i], st))) return e;
        return cudaSuccess;
    }
    if ((e = cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(int), st))) return e;
    for (int ph = 0; ph < 2; ph++) {
        if (ph == 1 && tensor(b)) {
            // each instance's force operand split once for its rhs group, then one launch over all items
            for (int i = 0; i < b->n; i++) {
                const fbc::Plan& P = b->plans[i]->p;
                if (P.K < 2) continue;
                if ((e = fbc::contract_tc_prep(P, P.d_fh, inst_rpc(b, i), b->n_rhs[i], 1, P.K - 1, st))) return e;
            }
            const fbc::Plan& P0 = b->plans[0]->p;
            const int wl = P0.wait_limit > 0 ? P0.wait_limit : (1 << 24);
            if ((e = fbc::launch_contract_tc_batch(b->precision, b->d_tc_jobs, b->d_con[1], (int)b->con_items[1].size(),
                                                   b->d_counter + 1, b->grid[1], b->smem_tc, wl, P0.d_status, st)))
                return e;
            continue;
        }
        if ((e = fbc::launch_batch_contract(b->precision, ph, b->d_cargs, b->d_nrhs, b->d_con[ph],
                                            (int)b->con_items[ph].size(), b->d_counter + ph, b->grid[ph],
                                            b->smem_con[ph], st)))
            return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int fbc_batch_create(fbc_plan* const* plans, int32_t n_plans, const double* const* f, double* const* u,
                     const int32_t* n_rhs, fbc_batch** out) {
    fbc::report_error(FBC_OK, "");
    if (!out) return bfail(FBC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || !f || !u || !n_rhs || n_plans < 1) return bfail(FBC_ERR_INVALID_ARG, "bad batch arguments");
    int prec = -1;
    for (int i = 0; i < n_plans; i++) {
        if (!plans[i]) return bfail(FBC_ERR_INVALID_ARG, "a plan is NULL");
        const fbc::Plan& P = plans[i]->p;
        if (P.host_only) return bfail(FBC_ERR_INVALID_ARG, "host-only plan in a batch");
        if (!P.tabulated) return bfail(FBC_ERR_NOT_TABULATED, "every plan of a batch must be tabulated");
        if (P.sur) return bfail(FBC_ERR_UNSUPPORTED, "a plan with a surrogate attached runs on its own");
        if (prec < 0) prec = P.precision;
        if (P.precision != prec) return bfail(FBC_ERR_INVALID_ARG, "all plans of a batch need the same precision");
        if (fbc::is_fft_precision(prec))
            return bfail(FBC_ERR_UNSUPPORTED, "batches run the dense per-mode contraction, not the in-plane FFT form");
        if (prec == FBC_PREC_BF16X6)
            return bfail(FBC_ERR_UNSUPPORTED, "BF16X6 plans run on their own, not in a batch");
        if (fbc::is_tensor_precision(prec) && fbc::contract_tc_smem(prec, P.W * P.H) > 227 * 1024)
            return bfail(FBC_ERR_UNSUPPORTED, "tensor-core contraction: an instance's sub-box exceeds shared memory");
        if (n_rhs[i] < 1 || n_rhs[i] > P.opt.max_rhs) return bfail(FBC_ERR_INVALID_ARG, "n_rhs outside [1, max_rhs]");
        if (!f[i] || !u[i]) return bfail(FBC_ERR_INVALID_ARG, "f or u of an instance is NULL");
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return bfail(FBC_ERR_INVALID_ARG, "a plan appears twice (its workspace would race)");
    }
    fbc_batch* b = new (std::nothrow) fbc_batch();
    if (!b) return bfail(FBC_ERR_OOM, "host allocation failed");
    b->n = n_plans;
    b->precision = prec;
    b->plans.assign(plans, plans + n_plans);
    b->n_rhs.assign(n_rhs, n_rhs + n_plans);
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    std::vector<fbc::LineArgs> la(n_plans);
    std::vector<fbc::ContractArgs> ca(n_plans);
    const int RB = fbc::batch_rhs_block();
    int max_L = 2;
    for (int i = 0; i < n_plans; i++) {
        const fbc::Plan& P = plans[i]->p;
        la[i] = fbc::make_line_args(P, f[i], u[i]);
        ca[i] = fbc::make_contract_args(P);
        max_L = std::max(max_L, P.L);
        for (int ph = 0; ph < 2; ph++)
            b->smem_con[ph] = std::max(b->smem_con[ph], fbc::batch_contract_smem_phase(prec, ph, P.W, P.H));
        const int R = n_rhs[i];
        const int NC = la[i].NC;
        for (int r = 0; r < R; r++) {
            for (int blk = 0; blk < P.NIpad / NC; blk++) b->fwd.push_back(make_int4(i, blk, r, 0));
            b->proj.push_back(make_int4(i, 0, r, 0));
            for (int blk = 0; blk < P.NPpad / NC; blk++) b->inv.push_back(make_int4(i, blk, r, 0));
            const size_t n_el = (size_t)P.n_p * P.L * 3;
            const int nch = (int)std::max<size_t>(1, std::min<size_t>(64, (n_el + 4095) / 4096));
            for (int c = 0; c < nch; c++) b->zm.push_back(make_int4(i, c, r, nch));
        }
        // contraction items; cost ~ pair-modes / measured rate of the tile kind
        const double per_tile = (double)P.n_tb * P.TA * P.TB;
        for (int k = 0; k < P.K; k++)
            for (int tA = 0; tA < P.n_ta; tA++) {
                if (fbc::is_tensor_precision(prec) && k > 0) {
                    continue;  // the tensor-core items are built below for the batch's rhs group
                } else if (fbc::is_tensor_precision(prec)) {  // k = 0 in double-float, as in a single plan
                    for (int r = 0; r < R; r++) b->con_items[0].push_back({make_int4(i, k, tA, r), per_tile / 130.0});
                } else if (prec == FBC_PREC_FP32 && k > 0) {
                    for (int rb = 0; rb < (R + RB - 1) / RB; rb++) {
                        const int cnt = std::min(RB, R - rb * RB);
                        b->con_items[1].push_back({make_int4(i, k, tA, rb), per_tile * cnt / 1500.0});
                    }
                } else if (prec == FBC_PREC_FP32) {  // k = 0 in double-float
                    for (int r = 0; r < R; r++) b->con_items[0].push_back({make_int4(i, k, tA, r), per_tile / 130.0});
                } else {
                    const double rate = (prec == FBC_PREC_F32X2) ? 130.0 : 34.0;
                    for (int r = 0; r < R; r++) b->con_items[1].push_back({make_int4(i, k, tA, r), per_tile / rate});
                }
            }
        b->pair_modes += (double)P.n_p * P.n_i * P.K * R;
    }
    if (fbc::is_tensor_precision(prec)) {
        b->rpc = 64;
        build_tc_items(b);
    }
    if (std::max(b->smem_con[0], b->smem_con[1]) > 227 * 1024) {
        free_batch(b);
        delete b;
        return bfail(FBC_ERR_UNSUPPORTED, "an instance's staged sub-box exceeds shared memory");
    }
    b->smem_line = 0;
    for (int i = 0; i < n_plans; i++)
        b->smem_line = std::max(b->smem_line, fbc::line_args_smem(la[i], fbc::line_fp32(prec)));
    std::vector<int> nr(b->n_rhs);
    cudaError_t e = cudaSuccess;
    if (!e) e = upload(&b->d_largs, la);
    if (!e) e = upload(&b->d_cargs, ca);
    if (!e) e = upload(&b->d_nrhs, nr);
    if (!e) e = upload(&b->d_fwd, b->fwd);
    if (!e) e = upload(&b->d_proj, b->proj);
    if (!e) e = upload(&b->d_inv, b->inv);
    if (!e) e = upload(&b->d_zm, b->zm);
    if (!e) e = upload(&b->d_con[0], ordered_items(b, 0, true));
    if (!e) e = upload(&b->d_con[1], ordered_items(b, 1, true));
    if (!e && tensor(b)) e = upload(&b->d_tc_jobs, b->tc_jobs);
    if (!e) e = cudaMalloc((void**)&b->d_counter, 2 * sizeof(int));
    if (!e) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e) {
        int st = bcuda(e, "batch setup");
        free_batch(b);
        delete b;
        return st;
    }
    for (int ph = 0; ph < 2; ph++) {
        // the tensor-core launch holds all of an SM's tensor memory: one CTA per SM
        b->occupancy[ph] = (ph == 1 && tensor(b)) ? 1 : fbc::batch_contract_occupancy_phase(prec, ph, b->smem_con[ph]);
        b->grid[ph] = b->occupancy[ph] * b->sm_count;
    }
    *out = b;
    return FBC_OK;
}

int fbc_batch_apply(fbc_batch* b, double alpha, double beta, uint32_t flags, void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!b) return bfail(FBC_ERR_INVALID_ARG, "batch is NULL");
    if (flags & ~(FBC_APPLY_PROJECT_NEUTRAL | FBC_APPLY_ZERO_MEAN_U | FBC_APPLY_NO_GRAPH))
        return bfail(FBC_ERR_INVALID_ARG, "unknown apply flags");
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return bfail(FBC_ERR_INVALID_ARG, "alpha/beta not finite");
    // the batch holds the plans' table pointers as they were at creation
    for (const fbc_plan* pl : b->plans)
        if (pl->p.sur || pl->p.precision != b->precision)
            return bfail(FBC_ERR_INVALID_ARG, "a plan changed precision or took a surrogate after the batch was made");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t gflags = flags & ~FBC_APPLY_NO_GRAPH;
    if (flags & FBC_APPLY_NO_GRAPH) {
        cudaError_t e = enqueue(b, alpha, beta, gflags, st);
        return e ? bcuda(e, "batched apply") : FBC_OK;
    }
    if (!b->graph_valid || b->g_alpha != alpha || b->g_beta != beta || b->g_flags != gflags) {
        if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
        if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
        if (e) return bcuda(e, "begin capture");
        cudaError_t e1 = enqueue(b, alpha, beta, gflags, b->cap);
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (e1) return bcuda(e1, "capture of the batched apply");
        if (e) return bcuda(e, "end capture");
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e) return bcuda(e, "graph instantiate");
        b->g_alpha = alpha, b->g_beta = beta, b->g_flags = gflags, b->graph_valid = true;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    return e ? bcuda(e, "graph launch") : FBC_OK;
}

int fbc_batch_autotune(fbc_batch* b, void* stream, double* best_ms) {
    fbc::report_error(FBC_OK, "");
    if (!b) return bfail(FBC_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return bfail(FBC_ERR_CUDA, "event creation failed");
    // the transforms run once so the contraction sees real inputs; the dominant launch (phase 1) is tuned
    cudaError_t e = fbc::launch_batch_line(0, b->d_largs, b->d_fwd, (int)b->fwd.size(), b->smem_line, 0, 0, 0, st, fbc::line_fp32(b->precision));
    const int ph = 1;
    if (!e && tensor(b)) {
        // candidates: per-instance launches, and the queue with each rhs group (largest first, then halves
        // that keep N = 2 rhs a multiple of 16) in both orders; each timed on the whole contraction
        int max_rpc = 1;
        for (int i = 0; i < b->n; i++) max_rpc = std::max(max_rpc, fbc::contract_tc_max_rpc(b->plans[i]->p));
        struct Cand { int form, rpc, lpt; };
        std::vector<Cand> cands = {{1, b->rpc, b->lpt}};
        for (int r = max_rpc; r >= 8; r /= 2)
            for (int lpt = 1; lpt >= 0; lpt--) cands.push_back({0, r, lpt});
        double best = 1e300;
        Cand bestc = cands[0];
        for (const Cand& c : cands) {
            b->tc_form = c.form, b->rpc = c.rpc, b->lpt = c.lpt;
            if (c.form == 0) {
                build_tc_items(b);
                if ((e = upload(&b->d_tc_jobs, b->tc_jobs))) break;
                if ((e = upload(&b->d_con[1], ordered_items(b, 1, c.lpt == 1)))) break;
            }
            float ms_sum = 0.0f;
            for (int rep = 0; rep < 2 && !e; rep++) {
                cudaEventRecord(e0, st);
                e = enqueue_contract(b, st);
                cudaEventRecord(e1, st);
                if (!e) e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1) ms_sum += ms;  // the first repetition warms caches
            }
            if (e) break;
            if (ms_sum < best) best = ms_sum, bestc = c;
        }
        if (!e) {
            b->tc_form = bestc.form, b->rpc = bestc.rpc, b->lpt = bestc.lpt;
            build_tc_items(b);
            e = upload(&b->d_tc_jobs, b->tc_jobs);
            if (!e) e = upload(&b->d_con[1], ordered_items(b, 1, bestc.lpt == 1));
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e) return bcuda(e, "autotune");
        b->graph_valid = false;
        if (best_ms) *best_ms = best;
        return FBC_OK;
    }
    double best = 1e300;
    int best_grid = b->grid[ph], best_lpt = b->lpt;
    const int occ = b->occupancy[ph];
    const int grids[] = {occ * b->sm_count, std::max(1, occ - 1) * b->sm_count, b->sm_count};
    for (int lpt = 1; lpt >= 0 && !e; lpt--) {
        if ((e = upload(&b->d_con[ph], ordered_items(b, ph, lpt == 1)))) break;
        for (int g : grids) {
            float ms_sum = 0.0f;
            for (int rep = 0; rep < 2 && !e; rep++) {
                if ((e = cudaMemsetAsync(b->d_counter + ph, 0, sizeof(int), st))) break;
                cudaEventRecord(e0, st);
                e = fbc::launch_batch_contract(b->precision, ph, b->d_cargs, b->d_nrhs, b->d_con[ph],
                                               (int)b->con_items[ph].size(), b->d_counter + ph, g, b->smem_con[ph], st);
                cudaEventRecord(e1, st);
                if (!e) e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1) ms_sum += ms;  // the first repetition warms caches
            }
            if (!e && ms_sum < best) best = ms_sum, best_grid = g, best_lpt = lpt;
        }
    }
    if (!e) e = upload(&b->d_con[ph], ordered_items(b, ph, best_lpt == 1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return bcuda(e, "autotune");
    b->grid[ph] = best_grid;
    b->lpt = best_lpt;
    b->graph_valid = false;
    if (best_ms) *best_ms = best;
    return FBC_OK;
}

int fbc_batch_info_get(const fbc_batch* b, fbc_batch_info* info) {
    fbc::report_error(FBC_OK, "");
    if (!b || !info) return bfail(FBC_ERR_INVALID_ARG, "batch or info is NULL");
    info->n_plans = b->n;
    info->precision = b->precision;
    info->n_contract_items = (int32_t)(b->con_items[0].size() + b->con_items[1].size());
    info->grid = b->grid[1];
    info->occupancy = b->occupancy[1];
    info->lpt_order = b->lpt;
    // forward, projection, contraction (one launch per non-empty phase), inverse, zero mean (when flagged)
    info->kernel_launches = 4 + (b->con_items[0].empty() ? 0 : 1) + (b->con_items[1].empty() ? 0 : 1);
    if (tensor(b) && b->tc_form == 1) {
        info->kernel_launches = 4;  // forward, projection, inverse, zero mean; per instance k = 0, split, tensor
        for (const fbc_plan* pl : b->plans) info->kernel_launches += pl->p.K > 1 ? 3 : 1;
    } else if (tensor(b)) {
        for (const fbc_plan* pl : b->plans) info->kernel_launches += pl->p.K > 1 ? 1 : 0;  // the force splits
    }
    info->smem_contract = tensor(b) ? b->smem_tc : b->smem_con[1];
    info->pair_modes = b->pair_modes;
    info->rhs_per_cta = tensor(b) ? inst_rpc(b, 0) : (b->precision == FBC_PREC_FP32 ? fbc::batch_rhs_block() : 1);
    info->launch_form = tensor(b) ? b->tc_form : 0;
    return FBC_OK;
}

void fbc_batch_destroy(fbc_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
    delete b;
}

}  // extern "C"
