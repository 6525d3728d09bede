// Batched AFMM products, host side: the plan of a batch (routes, operand
// buffers, TMA descriptors, balanced tile lists), its CUDA graph and the
// per-call pointer tables.  The kernels are in batched_kernels.cu.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <queue>
#include <vector>

#include "afmm_common.cuh"
#include "batched.cuh"
#include "tc_gemm.cuh"

namespace afmm {
namespace {

struct TileCost {
    int inst, tm, tn, cost;
};
bool cost_greater(const TileCost& a, const TileCost& b) { return a.cost > b.cost; }

template <typename T>
T* bump(char* base, size_t& top, size_t count) {
    top = (top + 255) / 256 * 256;
    T* p = reinterpret_cast<T*>(base + top);
    top += count * sizeof(T);
    return p;
}

struct BatchState {
    std::vector<afmm_desc> descs;
    int device = -1;
    std::vector<int> route;              // 1 tensor cores, 0 CUDA cores
    std::vector<int> tc_ids, simt_ids;   // instance indices per route
    // Host copies of the per-call tables (pointers refreshed each call).
    std::vector<GInst> ginst;
    std::vector<WJob> wjobs;
    std::vector<int> wjob_owner;         // instance of each widening job
    std::vector<int> wjob_which;         // 0: X, 1: Y
    std::vector<SimtJob> sjobs;
    std::vector<char> table_host;        // [GInst][WJob][SimtJob] packed
    // Device memory.
    char* mem = nullptr;
    size_t mem_bytes = 0;
    size_t table_bytes = 0;
    char* d_table = nullptr;
    GInst* d_ginst = nullptr;
    WJob* d_wjobs = nullptr;
    SimtJob* d_sjobs = nullptr;
    int* d_row_prefix = nullptr;
    int* d_tt_prefix = nullptr;
    int* d_row_job = nullptr;            // instance of each A-operand row
    int* d_tt_job = nullptr;             // instance of each 64 x 64 B tile
    int* d_wprefix = nullptr;
    int* d_sprefix = nullptr;
    int* d_cta_off = nullptr;
    TileRec* d_tiles = nullptr;
    int* d_flags = nullptr;
    int* d_status = nullptr;
    unsigned char* d_maps = nullptr;
    int rows_total = 0, tt_total = 0, wrows_total = 0, stiles_total = 0;
    int tc_grid = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int kernels = 0;
    ~BatchState() {
        if (exec) cudaGraphExecDestroy(exec);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
        if (mem) cudaFree(mem);
    }
};

std::mutex g_batch_mu;
std::list<std::unique_ptr<BatchState>> g_batches;   // most recent first
constexpr size_t kMaxCachedBatches = 4;

bool same_descs(const BatchState& b, int count, const afmm_desc* d, int dev) {
    return b.device == dev && (int)b.descs.size() == count &&
           std::memcmp(b.descs.data(), d, sizeof(afmm_desc) * (size_t)count) == 0;
}


afmm_status check_batch_desc(const afmm_desc& d) {
    if (d.n < 0 || d.reserved_ != 0 || d.target != AFMM_TARGET_FP32 ||
        d.z_dtype != AFMM_F32 || (d.kase != AFMM_CASE_A && d.kase != AFMM_CASE_B))
        return AFMM_ERR_INVALID_ARG;
    if ((d.ldx && d.ldx < d.n) || (d.ldy && d.ldy < d.n) || (d.ldz && d.ldz < d.n))
        return AFMM_ERR_INVALID_ARG;
    if (d.variant != AFMM_VARIANT_AUTO && d.variant != AFMM_VARIANT_SIMT_F32 &&
        d.variant != AFMM_VARIANT_TC_BF16X3 && d.variant != AFMM_VARIANT_TC_BF16X3_N128)
        return AFMM_ERR_UNSUPPORTED;
    const int rep = d.kase == AFMM_CASE_A ? d.y_dtype : d.x_dtype;
    const int real = d.kase == AFMM_CASE_A ? d.x_dtype : d.y_dtype;
    if (dtype_size(rep) == 0 || dtype_size(real) == 0 || rep == AFMM_F64 ||
        real == AFMM_E4M3)
        return AFMM_ERR_INVALID_ARG;
    return AFMM_OK;
}

afmm_status build_state(BatchState* b, int count, const afmm_desc* descs, int dev) {
    DeviceProps dp;
    AFMM_TRY(device_props(&dp));
    b->descs.assign(descs, descs + count);
    b->device = dev;
    const bool tc_ok = tc_available();
    for (int i = 0; i < count; ++i) {
        AFMM_TRY(check_batch_desc(descs[i]));
        int r = dispatch_route(descs[i]);
        if (r >= 1 && !tc_ok) {
            if (descs[i].variant == AFMM_VARIANT_TC_BF16X3 ||
                descs[i].variant == AFMM_VARIANT_TC_BF16X3_N128)
                return AFMM_ERR_UNSUPPORTED;
            r = 0;
        }
        if (descs[i].n == 0) r = -1;     // nothing to do
        b->route.push_back(r);
        if (r >= 1) b->tc_ids.push_back(i);
        else if (r == 0) b->simt_ids.push_back(i);
    }
    // ---- sizes
    const int ntc = (int)b->tc_ids.size();
    std::vector<int> row_prefix(ntc + 1, 0), tt_prefix(ntc + 1, 0);
    size_t opbytes = 0;
    for (int j = 0; j < ntc; ++j) {
        const int64_t n = descs[b->tc_ids[j]].n, ldk = (n + 7) / 8 * 8;
        const int sa = descs[b->tc_ids[j]].kase == AFMM_CASE_A ? 3 : 1;
        opbytes += ((size_t)sa * n * ldk * 2 + 255) / 256 * 256;
        opbytes += ((size_t)(4 - sa) * n * ldk * 2 + 255) / 256 * 256;
        row_prefix[j + 1] = row_prefix[j] + (int)n;
        const bool byte_tiles = descs[b->tc_ids[j]].kase == AFMM_CASE_A &&
                                dtype_size(descs[b->tc_ids[j]].y_dtype) == 1;
        tt_prefix[j + 1] = tt_prefix[j] + (int)g_transpose_blocks(n, byte_tiles);
    }
    // widening jobs for CUDA-core instances with non-FP32 operands
    std::vector<int> wprefix(1, 0);
    size_t wbytes = 0;
    // (an FP32 Rep-factor operand gets a check-only job: it is read in place)
    for (int i : b->simt_ids) {
        for (int which = 0; which < 2; ++which) {
            const int dt = which == 0 ? descs[i].x_dtype : descs[i].y_dtype;
            const bool rep = which == (descs[i].kase == AFMM_CASE_A ? 1 : 0);
            if (dt == AFMM_F32 && !rep) continue;
            WJob w{};
            w.n = descs[i].n;
            w.dtype = dt;
            w.rep = rep ? 1 : 0;
            b->wjobs.push_back(w);
            b->wjob_owner.push_back(i);
            b->wjob_which.push_back(which);
            wprefix.push_back(wprefix.back() + (int)w.n);
            if (dt != AFMM_F32) wbytes += ((size_t)w.n * w.n * 4 + 255) / 256 * 256;
        }
    }
    std::vector<int> sprefix(1, 0);
    for (int i : b->simt_ids) {
        SimtJob s{};
        s.M = s.N = s.K = descs[i].n;
        s.tiles_n = simt_tiles_n(s.N);
        b->sjobs.push_back(s);
        sprefix.push_back(sprefix.back() + simt_tiles(s.M, s.N));
    }
    // ---- tensor-core tiles, longest first onto the least loaded CTA
    std::vector<TileCost> tl;
    // (a tile's cost: its K steps times 4 for a 256-wide tile and 3 for a
    // 128-wide one -- a narrow tile costs three quarters of a wide one, not
    // half: measured, the batch with every tensor-core instance on 128-wide
    // tiles spent 1.49x the product time of the 256-wide batch on twice the
    // tiles -- plus a fixed share for the epilogue and the hand-over)
    for (int j = 0; j < ntc; ++j) {
        const int64_t n = descs[b->tc_ids[j]].n;
        const int bn = b->route[b->tc_ids[j]] == 2 ? 128 : GB_BN;
        const int tmn = (int)((n + GB_BM - 1) / GB_BM), tnn = (int)((n + bn - 1) / bn);
        const int cost = (int)((n + GB_BK - 1) / GB_BK) * (bn == 128 ? 3 : 4) + 16;
        for (int tm = 0; tm < tmn; ++tm)
            for (int tn = 0; tn < tnn; ++tn) tl.push_back({j, tm, tn, cost});
    }
    std::stable_sort(tl.begin(), tl.end(), cost_greater);
    const int grid = (int)std::min<size_t>(tl.size(), (size_t)dp.sm_count);
    std::vector<std::vector<TileRec>> per(grid);
    {
        using E = std::pair<long long, int>;
        std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
        for (int c = 0; c < grid; ++c) pq.push({0, c});
        for (const TileCost& t : tl) {
            E e = pq.top();
            pq.pop();
            per[e.second].push_back(TileRec{t.inst, t.tm, t.tn, 0});
            pq.push({e.first + t.cost, e.second});
        }
    }
    std::vector<int> cta_off(grid + 1, 0);
    std::vector<TileRec> tiles;
    for (int c = 0; c < grid; ++c) {
        cta_off[c + 1] = cta_off[c] + (int)per[c].size();
        tiles.insert(tiles.end(), per[c].begin(), per[c].end());
    }
    b->rows_total = row_prefix[ntc];
    b->tt_total = tt_prefix[ntc];
    std::vector<int> row_job(b->rows_total), tt_job(b->tt_total);
    for (int j = 0; j < ntc; ++j) {
        std::fill(row_job.begin() + row_prefix[j], row_job.begin() + row_prefix[j + 1], j);
        std::fill(tt_job.begin() + tt_prefix[j], tt_job.begin() + tt_prefix[j + 1], j);
    }
    b->wrows_total = wprefix.back();
    b->stiles_total = sprefix.back();
    b->tc_grid = grid;
    // ---- one device allocation
    b->ginst.resize(ntc);
    b->sjobs.resize(b->simt_ids.size());
    b->table_bytes = sizeof(GInst) * ntc + sizeof(WJob) * b->wjobs.size() +
                     sizeof(SimtJob) * b->sjobs.size();
    size_t top = 0;
    char* base = nullptr;
    for (int pass = 0; pass < 2; ++pass) {
        top = 0;
        b->d_maps = bump<unsigned char>(base, top, 2 * (size_t)ntc * 128);
        b->d_table = bump<char>(base, top, b->table_bytes);
        b->d_row_prefix = bump<int>(base, top, row_prefix.size());
        b->d_tt_prefix = bump<int>(base, top, tt_prefix.size());
        b->d_row_job = bump<int>(base, top, row_job.size() + 1);
        b->d_tt_job = bump<int>(base, top, tt_job.size() + 1);
        b->d_wprefix = bump<int>(base, top, wprefix.size());
        b->d_sprefix = bump<int>(base, top, sprefix.size());
        b->d_cta_off = bump<int>(base, top, cta_off.size());
        b->d_tiles = bump<TileRec>(base, top, tiles.size() + 1);
        b->d_flags = bump<int>(base, top, (size_t)ntc + 1);
        b->d_status = bump<int>(base, top, 64);
        char* ops = bump<char>(base, top, opbytes + wbytes);
        if (pass == 0) {
            b->mem_bytes = top;
            void* m = nullptr;
            AFMM_CUDA_TRY(cudaMalloc(&m, b->mem_bytes));
            b->mem = static_cast<char*>(m);
            base = b->mem;
            continue;
        }
        // operand buffers
        size_t o = 0;
        for (int j = 0; j < ntc; ++j) {
            const afmm_desc& d = descs[b->tc_ids[j]];
            const int64_t n = d.n, ldk = (n + 7) / 8 * 8;
            const int sa = d.kase == AFMM_CASE_A ? 3 : 1, sb = 4 - sa;
            GInst& g = b->ginst[j];
            std::memset(&g, 0, sizeof g);
            g.n = n;
            g.ldk = ldk;
            g.kind = d.kase == AFMM_CASE_A ? 0 : 1;
            g.x_dtype = d.x_dtype;
            g.y_dtype = d.y_dtype;
            g.ldx = d.ldx ? d.ldx : n;
            g.ldy = d.ldy ? d.ldy : n;
            g.ldz = d.ldz ? d.ldz : n;
            g.flag = j;
            g.bn = b->route[b->tc_ids[j]] == 2 ? 128 : GB_BN;
            g.A = ops + o;
            o += ((size_t)sa * n * ldk * 2 + 255) / 256 * 256;
            g.B = ops + o;
            o += ((size_t)sb * n * ldk * 2 + 255) / 256 * 256;
        }
        for (size_t w = 0; w < b->wjobs.size(); ++w) {
            if (b->wjobs[w].dtype == AFMM_F32) continue;      // check only
            b->wjobs[w].dst = reinterpret_cast<float*>(ops + o);
            o += ((size_t)b->wjobs[w].n * b->wjobs[w].n * 4 + 255) / 256 * 256;
        }
    }
    // tensor maps (host-encoded, copied to device)
    // 128-byte descriptors, 64-byte aligned, in a plain byte buffer.
    std::vector<unsigned char> mapbuf(2 * (size_t)ntc * 128 + 64);
    unsigned char* maps = mapbuf.data() +
                          ((64 - (reinterpret_cast<uintptr_t>(mapbuf.data()) & 63)) & 63);
    for (int j = 0; j < ntc; ++j) {
        // The three slices are always on the A side: Case A reads A = X
        // slices, B = Y^T; Case B computes Z^T = Y^T X^T, A = the Y^T slices
        // (buffer B), B = the X rows (buffer A).
        const GInst& g = b->ginst[j];
        void* a_side = g.kind == 0 ? g.A : g.B;
        void* b_side = g.kind == 0 ? g.B : g.A;
        AFMM_TRY(tc_encode_map(maps + 2 * j * 128, a_side, g.n, g.n, g.ldk, 3, GB_BM));
        AFMM_TRY(tc_encode_map(maps + (2 * j + 1) * 128, b_side, g.n, g.n, g.ldk, 1, g.bn));
    }
    auto up = [](void* dst, const void* src, size_t bytes) -> afmm_status {
        if (bytes) AFMM_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
        return AFMM_OK;
    };
    AFMM_TRY(up(b->d_maps, maps, 2 * (size_t)ntc * 128));
    AFMM_TRY(up(b->d_row_prefix, row_prefix.data(), row_prefix.size() * sizeof(int)));
    AFMM_TRY(up(b->d_tt_prefix, tt_prefix.data(), tt_prefix.size() * sizeof(int)));
    AFMM_TRY(up(b->d_row_job, row_job.data(), row_job.size() * sizeof(int)));
    AFMM_TRY(up(b->d_tt_job, tt_job.data(), tt_job.size() * sizeof(int)));
    AFMM_TRY(up(b->d_wprefix, wprefix.data(), wprefix.size() * sizeof(int)));
    AFMM_TRY(up(b->d_sprefix, sprefix.data(), sprefix.size() * sizeof(int)));
    AFMM_TRY(up(b->d_cta_off, cta_off.data(), cta_off.size() * sizeof(int)));
    AFMM_TRY(up(b->d_tiles, tiles.data(), tiles.size() * sizeof(TileRec)));
    AFMM_CUDA_TRY(cudaMemset(b->d_status, 0, 64 * sizeof(int)));
    b->d_ginst = reinterpret_cast<GInst*>(b->d_table);
    b->d_wjobs = reinterpret_cast<WJob*>(b->d_table + sizeof(GInst) * ntc);
    b->d_sjobs = reinterpret_cast<SimtJob*>(b->d_table + sizeof(GInst) * ntc +
                                           sizeof(WJob) * b->wjobs.size());
    b->table_host.resize(b->table_bytes);
    return AFMM_OK;
}

// The launches of one batch call, in stream order on `st` (tensor-core
// branch) and `side` (CUDA-core branch), joined back into `st`.
afmm_status enqueue(BatchState* b, cudaStream_t st, cudaStream_t side,
                    cudaEvent_t fork, cudaEvent_t join, int* kernels) {
    const int ntc = (int)b->tc_ids.size();
    int k = 0;
    AFMM_CUDA_TRY(cudaEventRecord(fork, st));
    AFMM_CUDA_TRY(cudaStreamWaitEvent(side, fork, 0));
    if (ntc > 0) {
        AFMM_TRY(launch_batch_convert(b->d_ginst, b->d_row_prefix, b->d_row_job,
                                      b->d_tt_prefix, b->d_tt_job, ntc, b->rows_total,
                                      b->tt_total, b->d_flags, b->d_status, st));
        AFMM_TRY(launch_batch_tc(b->d_ginst, b->d_maps, b->d_cta_off,
                                 reinterpret_cast<const int*>(b->d_tiles), b->tc_grid,
                                 b->d_flags, b->d_status, st));
        k += 3;
    }
    const int nw = (int)b->wjobs.size(), ns = (int)b->sjobs.size();
    if (nw > 0) {
        AFMM_TRY(launch_batch_widen(b->d_wjobs, b->d_wprefix, nw, b->wrows_total,
                                    b->d_status, side));
        ++k;
    }
    if (ns > 0) {
        AFMM_TRY(launch_simt_f32_grouped(b->d_sjobs, b->d_sprefix, ns, b->stiles_total,
                                         side));
        ++k;
    }
    AFMM_CUDA_TRY(cudaEventRecord(join, side));
    AFMM_CUDA_TRY(cudaStreamWaitEvent(st, join, 0));
    *kernels = k;
    return AFMM_OK;
}

afmm_status capture(BatchState* b) {
    AFMM_CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    AFMM_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    AFMM_CUDA_TRY(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
    cudaStream_t cap;
    AFMM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    afmm_status rc = AFMM_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        rc = AFMM_ERR_CUDA;
    } else {
        const int64_t l0 = launch_counter();
        rc = enqueue(b, cap, b->side, b->fork, b->join, &b->kernels);
        count_launches(-(int)(launch_counter() - l0));   // counted per replay
        if (cudaStreamEndCapture(cap, &graph) != cudaSuccess) rc = AFMM_ERR_CUDA;
    }
    if (rc == AFMM_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess)
        rc = AFMM_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    cudaGetLastError();
    return rc;
}

}  // namespace

// ---------------------------------------------------------- dispatch model
// Route of a forced batched variant (-1: not a batched route).
static int route_of_variant(int v) {
    switch (v) {
        case AFMM_VARIANT_SIMT_F32: return 0;
        case AFMM_VARIANT_TC_BF16X3: return 1;
        case AFMM_VARIANT_TC_BF16X3_N128: return 2;
        default: return -1;
    }
}

struct DispatchModel {
    afmm_mlp_shape shape{};
    std::vector<float> params, mean, scale;
    std::vector<int> variant_of_output;
};
static std::mutex g_model_mu;
static std::unique_ptr<DispatchModel> g_model;

static void features_of(const afmm_desc& d, float* f) {
    const double n = (double)(d.n > 0 ? d.n : 1);
    const bool a = d.kase == AFMM_CASE_A;
    const double d1 = d.d1 >= 0.0 ? d.d1 : 1.0, d2 = d.d2 >= 0.0 ? d.d2 : 1.0;
    const double mu = d.mu_prime >= 0.0 ? d.mu_prime : 1.0;
    const double dbase = a ? d1 : d2, drep = a ? d2 : d1;
    f[0] = (float)std::log2(n);
    f[1] = (float)dbase;
    f[2] = (float)drep;
    f[3] = (float)std::log2(1.0 + mu);
    f[4] = a ? 0.f : 1.f;
    f[5] = (float)std::log2(1.0 + mu * d1 * d2 * n * n * n);
    f[6] = (float)(3.0 * std::log2(n));
    f[7] = (float)std::pow(1.0 - dbase, 8.0);
    f[8] = (float)(std::ceil(n / 256.0) * 256.0 / n);
    f[9] = (float)(std::ceil(n / 128.0) * 128.0 / n);
}

// Variant with the smallest predicted time, or -1 without a model.
static int model_route(const afmm_desc& d) {
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!g_model) return -1;
    const DispatchModel& m = *g_model;
    const int F = m.shape.features, H = m.shape.hidden, V = m.shape.outputs;
    std::vector<double> x(F), h1(H), h2(H);
    float f[AFMM_DISPATCH_FEATURES];
    features_of(d, f);
    for (int i = 0; i < F; ++i)
        x[i] = ((i < AFMM_DISPATCH_FEATURES ? f[i] : 0.f) - m.mean[i]) / m.scale[i];
    const float* W1 = m.params.data();
    const float* b1 = W1 + (size_t)F * H;
    const float* W2 = b1 + H;
    const float* b2 = W2 + (size_t)H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + (size_t)H * V;
    for (int o = 0; o < H; ++o) {
        double s = b1[o];
        for (int i = 0; i < F; ++i) s += x[i] * W1[(size_t)i * H + o];
        h1[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < H; ++o) {
        double s = b2[o];
        for (int i = 0; i < H; ++i) s += h1[i] * W2[(size_t)i * H + o];
        h2[o] = s > 0.0 ? s : 0.0;
    }
    int best = -1;
    double bestv = 0.0;
    for (int o = 0; o < V; ++o) {
        double s = b3[o];
        for (int i = 0; i < H; ++i) s += h2[i] * W3[(size_t)i * V + o];
        if (best < 0 || s < bestv) {
            best = o;
            bestv = s;
        }
    }
    return m.variant_of_output[best];
}


afmm_status dispatch_features(const afmm_desc& d, float* out) {
    features_of(d, out);
    return AFMM_OK;
}

afmm_status set_dispatch_model(const afmm_mlp_shape* s, const float* params,
                               const float* mean, const float* scale,
                               const int32_t* variants) {
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!params) {
        g_model.reset();
        return AFMM_OK;
    }
    if (!s || !mean || !scale || !variants || s->features <= 0 ||
        s->features > AFMM_DISPATCH_FEATURES || s->hidden <= 0 || s->outputs <= 0)
        return AFMM_ERR_INVALID_ARG;
    auto m = std::make_unique<DispatchModel>();
    m->shape = *s;
    const size_t np = (size_t)mlp_param_count(*s);
    m->params.assign(params, params + np);
    m->mean.assign(mean, mean + s->features);
    m->scale.assign(scale, scale + s->features);
    for (int i = 0; i < s->features; ++i)
        if (!(m->scale[i] > 0.f)) return AFMM_ERR_INVALID_ARG;
    for (int o = 0; o < s->outputs; ++o) {
        const int r = route_of_variant(variants[o]);
        if (r < 0) return AFMM_ERR_INVALID_ARG;
        m->variant_of_output.push_back(r);
    }
    g_model = std::move(m);
    return AFMM_OK;
}

int dispatch_route(const afmm_desc& d) {
    const int forced = route_of_variant(d.variant);
    if (forced >= 0) return forced;
    const int r = model_route(d);
    return r >= 0 ? r : batch_rule_route(d);
}


int batch_rule_route(const afmm_desc& d) {
    // Tensor cores unless the Base factor is so sparse that the CUDA-core
    // zero-skip removes most of the dense work (a whole 8-row group of Base
    // values zero at a given k happens with probability (1 - d)^8).
    const double dbase = d.kase == AFMM_CASE_A ? d.d1 : d.d2;
    if (d.n < 32) return 0;
    if (dbase >= 0.0 && dbase < 0.02) return 0;
    return 1;
}

afmm_status batched_run(int count, const afmm_desc* descs, const void* const* X,
                        const void* const* Y, void* const* Z, void* stream,
                        int* kernels_out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return AFMM_ERR_NO_DEVICE;
    }
    for (int i = 0; i < count; ++i)
        if (descs[i].n > 0 && (!X[i] || !Y[i] || !Z[i])) return AFMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchState* b = nullptr;
    for (auto it = g_batches.begin(); it != g_batches.end(); ++it)
        if (same_descs(**it, count, descs, dev)) {
            g_batches.splice(g_batches.begin(), g_batches, it);
            b = g_batches.front().get();
            break;
        }
    if (!b) {
        auto nb = std::make_unique<BatchState>();
        AFMM_TRY(build_state(nb.get(), count, descs, dev));
        AFMM_TRY(capture(nb.get()));
        g_batches.push_front(std::move(nb));
        while (g_batches.size() > kMaxCachedBatches) g_batches.pop_back();
        b = g_batches.front().get();
    }
    // Refresh the pointer tables.
    for (size_t j = 0; j < b->tc_ids.size(); ++j) {
        const int i = b->tc_ids[j];
        b->ginst[j].X = X[i];
        b->ginst[j].Y = Y[i];
        b->ginst[j].Z = static_cast<float*>(Z[i]);
    }
    for (size_t w = 0; w < b->wjobs.size(); ++w) {
        const int i = b->wjob_owner[w];
        const afmm_desc& d = descs[i];
        b->wjobs[w].src = b->wjob_which[w] == 0 ? X[i] : Y[i];
        b->wjobs[w].lds = b->wjob_which[w] == 0 ? (d.ldx ? d.ldx : d.n) : (d.ldy ? d.ldy : d.n);
    }
    for (size_t s = 0; s < b->simt_ids.size(); ++s) {
        const int i = b->simt_ids[s];
        const afmm_desc& d = descs[i];
        SimtJob& j = b->sjobs[s];
        j.A = static_cast<const float*>(X[i]);
        j.lda = d.ldx ? d.ldx : d.n;
        j.B = static_cast<const float*>(Y[i]);
        j.ldb = d.ldy ? d.ldy : d.n;
        for (size_t w = 0; w < b->wjobs.size(); ++w)
            if (b->wjob_owner[w] == i && b->wjobs[w].dst) {
                if (b->wjob_which[w] == 0) { j.A = b->wjobs[w].dst; j.lda = d.n; }
                else { j.B = b->wjobs[w].dst; j.ldb = d.n; }
            }
        j.C = static_cast<float*>(Z[i]);
        j.ldc = d.ldz ? d.ldz : d.n;
        auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
        j.vec = (j.lda % 4 == 0) && (j.ldb % 4 == 0) && (j.ldc % 4 == 0) && al(j.A) &&
                al(j.B) && al(j.C);
    }
    char* h = b->table_host.data();
    std::memcpy(h, b->ginst.data(), sizeof(GInst) * b->ginst.size());
    h += sizeof(GInst) * b->ginst.size();
    std::memcpy(h, b->wjobs.data(), sizeof(WJob) * b->wjobs.size());
    h += sizeof(WJob) * b->wjobs.size();
    std::memcpy(h, b->sjobs.data(), sizeof(SimtJob) * b->sjobs.size());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Pageable source: the copy is staged before this call returns, so the
    // host table can be refilled by the next call at once.
    if (b->table_bytes)
        AFMM_CUDA_TRY(cudaMemcpyAsync(b->d_table, b->table_host.data(), b->table_bytes,
                                      cudaMemcpyHostToDevice, st));
    AFMM_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    count_launches(b->kernels);
    if (kernels_out) *kernels_out = b->kernels;
    return AFMM_OK;
}

afmm_status batched_status(int count, const afmm_desc* descs, int* out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return AFMM_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& b : g_batches)
        if (same_descs(*b, count, descs, dev)) {
            int h[2] = {0, 0};
            AFMM_CUDA_TRY(cudaMemcpy(&h[0], b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
            *out = h[0];
            // A reported error is cleared, so the next call starts clean.
            if (h[0] != 0)
                AFMM_CUDA_TRY(cudaMemcpy(b->d_status, &h[1], sizeof(int),
                                         cudaMemcpyHostToDevice));
            return AFMM_OK;
        }
    return AFMM_ERR_INVALID_ARG;
}

void batched_clear_cache() {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batches.clear();
}

}  // namespace afmm
