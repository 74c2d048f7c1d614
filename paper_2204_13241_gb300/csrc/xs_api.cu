// C ABI of libxs: argument checking, workspace, frame streaming and launches.
// The operations themselves are defined in include/xs_api.h with citations.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "xs_api.h"
#include "xs_internal.h"

using namespace xs;

namespace xs {
thread_local int64_t tl_kernel_launches = 0;
}

namespace {
thread_local std::string g_last_error;
}

void xs::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {

xs_status fail(xs_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define XS_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(XS_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                             \
    } while (0)

// inverse of a row-major 3x3 by the adjugate; false when singular
bool invert3(const double* h, double* out) {
    double adj[9];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            // cofactor of element (c, r) goes to adj[r][c]
            const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
            adj[r * 3 + c] = h[r1 * 3 + c1] * h[r2 * 3 + c2] - h[r1 * 3 + c2] * h[r2 * 3 + c1];
        }
    }
    const double det = h[0] * adj[0] + h[1] * adj[3] + h[2] * adj[6];
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    for (int i = 0; i < 9; ++i) out[i] = adj[i] / det;
    return true;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// odd multiplier near 0.618 n coprime with n: k -> k*a mod n visits the atom
// runs far apart in input order (a bijection on [0, n))
int64_t coprime_stride(int64_t n) {
    if (n <= 2) return 1;
    int64_t a = (int64_t)(0.6180339887498949 * (double)n) | 1;
    while (gcd64(a, n) != 1) a += 2;
    return a % n == 0 ? 1 : a;
}

bool is_ortho(const double* hinv) {
    return hinv[1] == 0.0 && hinv[2] == 0.0 && hinv[3] == 0.0 && hinv[5] == 0.0 && hinv[6] == 0.0 && hinv[7] == 0.0;
}

// shape bucket of the tuner's cache: atoms by powers of two (the choice of
// tile kind and chunk length hardly depends on the exact count), the
// contracted grid's extents and the precision
std::tuple<int, int, int, int, int> tc_bucket(int64_t n_pad, const GridDesc& g, int prec) {
    int lg = 0;
    while (lg < 62 && ((int64_t)1 << (lg + 1)) <= n_pad) ++lg;
    return std::make_tuple(lg, g.nx, g.ny, g.nz, prec);
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct xs_context {
    int device = 0;
    int num_sms = 0;
    xs_allocator alloc{};
    bool has_alloc = false;
    void* ws = nullptr;  // grow-only workspace
    size_t ws_bytes = 0;
    int* d_err = nullptr;
    int64_t timeout_ns = 2000000000LL;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
    // tuner results per shape bucket (tc_bucket): tile kind and chunk length
    struct TcChoice {
        int kind;
        int chunk;
    };
    std::map<std::tuple<int, int, int, int, int>, TcChoice> tuned;
    bool exact_tables = false;  // tensor-core tables from FP64 sincospi per entry
    // small device-side tables, one slot per caller tag, re-uploaded only
    // when their content changes (so repeated calls enqueue no host copies)
    struct ConstSlot {
        std::vector<char> key;
        void* dev = nullptr;
        size_t bytes = 0;
    };
    std::map<std::string, ConstSlot> consts;
    // tracing
    struct ProfRec {
        std::string name;
        cudaEvent_t a, b;
        int64_t kernels;
    };
    struct Graph {
        cudaGraphExec_t exec;
        int64_t kernels;
    };
    std::map<std::string, Graph> graphs;  // captured batched launches
    void clear_graphs() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
        graphs.clear();
    }
    bool prof_on = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    int64_t launches = 0;

    cudaEvent_t take_event() {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }

    void* raw_alloc(size_t bytes) {
        if (has_alloc) return alloc.alloc(bytes, alloc.ctx);
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void raw_free(void* p) {
        if (!p) return;
        if (has_alloc)
            alloc.free(p, alloc.ctx);
        else
            cudaFree(p);
    }
};

namespace {

// Ensures `bytes` of workspace; growing synchronizes the device first because
// earlier work may still read the old block.
xs_status ensure_ws(xs_context* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return XS_OK;
    if (ctx->ws) {
        XS_CUDA(cudaDeviceSynchronize());
        ctx->clear_graphs();  // captured launches point into the old block
        ctx->raw_free(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    ctx->ws = ctx->raw_alloc(want);
    if (!ctx->ws) return fail(XS_ERR_NO_MEMORY, "workspace allocation of %zu bytes failed", want);
    ctx->ws_bytes = want;
    return XS_OK;
}

// Uploads a blob of small tables unless the same bytes are already resident.
xs_status upload_const(xs_context* ctx, const char* tag, const std::vector<char>& blob, cudaStream_t st,
                       void** dev) {
    xs_context::ConstSlot& slot = ctx->consts[tag];
    if (slot.dev && blob == slot.key) {
        *dev = slot.dev;
        return XS_OK;
    }
    // earlier launches on the stream may still read the old tables
    XS_CUDA(cudaStreamSynchronize(st));
    if (blob.size() > slot.bytes) {
        ctx->clear_graphs();  // captured launches may point into the old tables
        ctx->raw_free(slot.dev);
        slot.bytes = blob.size() + 4096;
        slot.dev = ctx->raw_alloc(slot.bytes);
        if (!slot.dev) {
            slot.bytes = 0;
            return fail(XS_ERR_NO_MEMORY, "table allocation failed");
        }
    }
    XS_CUDA(cudaMemcpy(slot.dev, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    slot.key = blob;
    *dev = slot.dev;
    return XS_OK;
}

template <class T>
size_t push(std::vector<char>& blob, const T* data, size_t n) {
    size_t off = round_up((int64_t)blob.size(), 256);
    blob.resize(off + n * sizeof(T));
    if (n) std::memcpy(blob.data() + off, data, n * sizeof(T));
    return off;
}

xs_status check_grid(const xs_qgrid* g) {
    if (!g) return fail(XS_ERR_INVALID_ARG, "grid is NULL");
    if (g->nx < 0 || g->ny < 0 || g->nz < 0) return fail(XS_ERR_INVALID_ARG, "negative grid extent");
    if (g->nx > 65536 || g->ny > 65536 || g->nz > 65536) return fail(XS_ERR_INVALID_ARG, "grid extent too large");
    return XS_OK;
}

GridDesc to_desc(const xs_qgrid* g) { return GridDesc{g->nx0, g->nx, g->ny0, g->ny, g->nz0, g->nz}; }

// Runs one launch_* call: counts its kernels and, when tracing, brackets it
// with events on the launching stream.
// Every launch group runs inside an NVTX range of its name ("phase", "tc",
// ...), so a timeline tool shows the stages of a call; with no tool attached
// the header-only NVTX calls return at once.
template <class F>
cudaError_t traced(xs_context* ctx, const char* name, cudaStream_t st, F&& launch) {
    struct NvtxRange {
        explicit NvtxRange(const char* n) { nvtxRangePushA(n); }
        ~NvtxRange() { nvtxRangePop(); }
    } range(name);
    const int64_t before = tl_kernel_launches;
    cudaEvent_t a = nullptr;
    if (ctx->prof_on) {
        a = ctx->take_event();
        if (a) cudaEventRecord(a, st);
    }
    const cudaError_t e = launch();
    const int64_t n = tl_kernel_launches - before;
    ctx->launches += n;
    if (ctx->prof_on && a) {
        cudaEvent_t b = ctx->take_event();
        if (b) {
            cudaEventRecord(b, st);
            ctx->prof.push_back({name, a, b, n});
        } else {
            ctx->event_pool.push_back(a);
        }
    }
    return e;
}

}  // namespace

extern "C" {

const char* xs_version(void) { return "xs 0.1 (sm_103a)"; }

const char* xs_last_error(void) { return g_last_error.c_str(); }

xs_status xs_context_create(const xs_allocator* allocator, xs_context** out) {
    if (!out) return fail(XS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(XS_ERR_INVALID_ARG, "allocator needs both alloc and free");
    xs_context* ctx = new xs_context();
    if (allocator) {
        ctx->alloc = *allocator;
        ctx->has_alloc = true;
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(XS_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    ctx->d_err = static_cast<int*>(ctx->raw_alloc(256));
    if (!ctx->d_err) {
        delete ctx;
        return fail(XS_ERR_NO_MEMORY, "error word allocation failed");
    }
    e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_consumed[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        xs_context_destroy(ctx);
        return fail(XS_ERR_CUDA, "context setup failed: %s", cudaGetErrorString(e));
    }
    *out = ctx;
    return XS_OK;
}

xs_status xs_context_destroy(xs_context* ctx) {
    if (!ctx) return XS_OK;
    cudaDeviceSynchronize();
    ctx->clear_graphs();
    ctx->raw_free(ctx->ws);
    ctx->raw_free(ctx->d_err);
    for (auto& kv : ctx->consts) ctx->raw_free(kv.second.dev);
    for (int i = 0; i < 2; ++i) {
        if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
        if (ctx->ev_consumed[i]) cudaEventDestroy(ctx->ev_consumed[i]);
    }
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (auto& r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
    return XS_OK;
}

xs_status xs_set_table_builder(xs_context* ctx, int32_t mode) {
    if (!ctx || (mode != 0 && mode != 1)) return fail(XS_ERR_INVALID_ARG, "table builder mode is 0 or 1");
    ctx->exact_tables = mode == 1;
    return XS_OK;
}

xs_status xs_set_wait_timeout_ns(xs_context* ctx, int64_t ns) {
    if (!ctx || ns <= 0) return fail(XS_ERR_INVALID_ARG, "bad context or timeout");
    ctx->timeout_ns = ns;
    return XS_OK;
}

xs_status xs_profile_enable(xs_context* ctx, int32_t on) {
    if (!ctx) return fail(XS_ERR_INVALID_ARG, "context is NULL");
    ctx->prof_on = on != 0;
    return XS_OK;
}

xs_status xs_profile_read(xs_context* ctx, const char* prefix, double* total_ms, int64_t* launches) {
    if (!ctx || !total_ms || !launches) return fail(XS_ERR_INVALID_ARG, "missing argument");
    const std::string pre = prefix ? prefix : "";
    double ms = 0.0;
    int64_t n = 0;
    xs_status st = XS_OK;
    std::vector<xs_context::ProfRec> keep;
    for (auto& r : ctx->prof) {
        if (r.name.compare(0, pre.size(), pre) != 0) {
            keep.push_back(r);
            continue;
        }
        float e = 0.0f;
        cudaError_t err = cudaEventSynchronize(r.b);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&e, r.a, r.b);
        if (err != cudaSuccess && st == XS_OK) st = fail(XS_ERR_CUDA, "profile event: %s", cudaGetErrorString(err));
        ms += e;
        n += r.kernels;
        ctx->event_pool.push_back(r.a);
        ctx->event_pool.push_back(r.b);
    }
    ctx->prof.swap(keep);
    *total_ms = ms;
    *launches = n;
    return st;
}

xs_status xs_launch_count(xs_context* ctx, int64_t* count) {
    if (!ctx || !count) return fail(XS_ERR_INVALID_ARG, "missing argument");
    *count = ctx->launches;
    return XS_OK;
}

xs_status xs_sync_status(xs_context* ctx, void* cuda_stream) {
    if (!ctx) return fail(XS_ERR_INVALID_ARG, "context is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    XS_CUDA(cudaStreamSynchronize(st));
    int word = 0;
    XS_CUDA(cudaMemcpy(&word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    XS_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
    if (word & kDevErrTimeout) return fail(XS_ERR_TIMEOUT, "a kernel wait timed out (device error word %d)", word);
    if (word & kDevErrNonFinite) return fail(XS_ERR_NUMERIC, "non-finite form factor, or a position that is non-finite or more than 2^18 cells from the origin (device error word %d)", word);
    if (word & kDevErrBounds) return fail(XS_ERR_BOUNDS, "a bounds check failed and its access was skipped (device error word %d)", word);
    return XS_OK;
}

// --------------------------------------------------------------------------
// intensity
// --------------------------------------------------------------------------

static xs_status intensity_impl(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid,
                                xs_precision prec, float* I_out, float* amp_out, cudaStream_t st,
                                int chunk_override, int kind_override = -1) {
    if (!ctx || !traj || !I_out) return fail(XS_ERR_INVALID_ARG, "context, trajectory and I_out are required");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (prec != XS_PREC_FP32_DIRECT && prec != XS_PREC_SPLIT_FP16 && prec != XS_PREC_SPLIT_BF16 &&
        prec != XS_PREC_FP32_FACTORED)
        return fail(XS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (traj->n_atoms < 0 || traj->n_frames < 0) return fail(XS_ERR_INVALID_ARG, "negative atom or frame count");
    if (traj->n_atoms > (int64_t)1 << 31) return fail(XS_ERR_INVALID_ARG, "more than 2^31 atoms");
    if (traj->n_atoms > 0 && traj->n_frames > 0 && (!traj->pos || !traj->f))
        return fail(XS_ERR_INVALID_ARG, "positions or form factors are NULL");
    double hinv[9];
    if (!invert3(traj->box.h, hinv)) return fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    const GridDesc g = to_desc(grid);
    const int64_t P = g.pixels();
    const int64_t T = traj->n_frames;
    if (P == 0 || T == 0) return XS_OK;
    const bool use_tc = prec == XS_PREC_SPLIT_FP16 || prec == XS_PREC_SPLIT_BF16;
    const bool factored = prec == XS_PREC_FP32_FACTORED;
    if (use_tc && !tc_supported(g)) return fail(XS_ERR_UNSUPPORTED, "grid not supported by the tensor-core path");

    const bool out_dev = is_device_ptr(I_out) && (!amp_out || is_device_ptr(amp_out));
    const bool pos_host = traj->pos_on_host != 0;
    if (traj->n_atoms > 0) {
        if (pos_host == is_device_ptr(traj->pos))
            return fail(XS_ERR_INVALID_ARG, "pos_on_host=%d does not match where pos lives", (int)traj->pos_on_host);
    }
    Mat3 hm;
    for (int i = 0; i < 9; ++i) hm.a[i] = hinv[i];
    const int64_t N = traj->n_atoms;
    const int64_t n_pad = round_up(N > 0 ? N : 1, 64);
    // with device outputs the tensor path may contract a half grid and fill
    // the rest by I(-q) = I(q) (real form factors), where that needs fewer tiles
    GridDesc gh = g;
    const int half_axis = (use_tc && out_dev && N > 0) ? friedel_half_grid(g, gh) : -1;
    const GridDesc gc = half_axis >= 0 ? gh : g;  // the contraction's grid
    PhaseOpts popt;
    popt.ortho = is_ortho(hinv);
    popt.need_z = !(gc.nz == 1 && gc.nz0 == 0);
    popt.perm_mul = use_tc ? coprime_stride(n_pad / kPermRun) : 1;

    // frames per chunk: records and (for host positions) staged positions
    const size_t rec_per_frame = (size_t)n_pad * sizeof(AtomRec);
    const size_t pos_per_frame = (size_t)N * 3 * sizeof(float);
    const size_t cap = (size_t)6 << 30;
    int64_t fchunk = T;
    if ((size_t)T * rec_per_frame > cap) fchunk = std::max<int64_t>(1, (int64_t)(cap / rec_per_frame));
    if (pos_host) fchunk = std::min<int64_t>(fchunk, std::max<int64_t>(1, (int64_t)((size_t)1 << 30) / std::max<size_t>(pos_per_frame, 1)));
    if (fchunk > 65535) fchunk = 65535;
    // chunks (first frame, frames).  Streamed host positions on the tensor
    // path start with about 64 MB and double up to fchunk: only the first copy
    // is exposed, and each later copy (twice the frames) hides behind the
    // previous chunk's kernels as long as the host link moves a frame's
    // positions faster than the kernels take for half a frame
    std::vector<std::pair<int64_t, int64_t>> chunks;
    {
        int64_t nf = fchunk;
        if (pos_host && use_tc)
            nf = std::min<int64_t>(fchunk, std::max<int64_t>(1, (int64_t)((size_t)64 << 20) /
                                                                   std::max<size_t>(pos_per_frame, 1)));
        for (int64_t t0 = 0; t0 < T;) {
            const int64_t n = std::min(nf, T - t0);
            chunks.emplace_back(t0, n);
            t0 += n;
            nf = std::min(fchunk, 2 * nf);
        }
    }

    DirectPlan dplan{};
    FactoredPlan fplan{};
    int tc_pairs = 0;
    int chunk_stages = kDefaultChunkStages;
    int tile_kind = kTcTile128;
    if (use_tc) {
        // half grids are planned on 128 x 128 tiles; otherwise the tuned tile
        // kind of this shape, else the default rule
        tile_kind = half_axis >= 0 ? kTcTile128 : tc_default_kind(gc);
        auto it = ctx->tuned.find(tc_bucket(n_pad, gc, (int)prec));
        if (it != ctx->tuned.end()) {
            chunk_stages = it->second.chunk;
            if (half_axis < 0) tile_kind = it->second.kind;
        }
        if (chunk_override > 0) chunk_stages = chunk_override;
        if (kind_override >= 0 && half_axis < 0) tile_kind = kind_override;
        tc_pairs = tc_pair_capacity(ctx->num_sms, tile_kind);
    } else if (factored) {
        fplan = plan_factored(n_pad, fchunk, g, ctx->num_sms);
    } else {
        dplan = plan_direct(n_pad, fchunk, g, ctx->num_sms);
    }

    // workspace layout
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = round_up((int64_t)off, 256);
        off = o + bytes;
        return o;
    };
    const size_t o_rec = carve((size_t)fchunk * rec_per_frame);
    const size_t o_part =
        carve(use_tc ? tc_scratch_bytes(tc_pairs) : (factored ? fplan.partial_bytes : dplan.partial_bytes));
    auto split_of = [&](int64_t nf) {
        return tc_split_plan(tc_units(tc_traj(nullptr, n_pad, nf, gc, nullptr, nullptr, tile_kind)), tc_pairs,
                             (int)(n_pad / tc_atom_multiple()), chunk_stages);
    };
    size_t split_bytes = 0;
    if (use_tc)
        for (const auto& ch : chunks) split_bytes = std::max(split_bytes, tc_split_bytes(split_of(ch.second)));
    const size_t o_split = carve(split_bytes);
    const size_t o_pos0 = carve(pos_host ? (size_t)fchunk * pos_per_frame : 0);
    const size_t o_pos1 = carve(pos_host ? (size_t)fchunk * pos_per_frame : 0);
    const size_t o_f = carve(pos_host ? (size_t)N * sizeof(float) : 0);
    const size_t o_I = carve(out_dev ? 0 : (size_t)fchunk * P * sizeof(float));
    const size_t o_amp = carve(out_dev || !amp_out ? 0 : (size_t)fchunk * P * 2 * sizeof(float));
    const size_t o_half = carve(half_axis >= 0 ? (size_t)fchunk * gh.pixels() * sizeof(float) : 0);
    const size_t o_half_amp = carve(half_axis >= 0 && amp_out ? (size_t)fchunk * gh.pixels() * 2 * sizeof(float) : 0);
    s = ensure_ws(ctx, off + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    AtomRec* rec = reinterpret_cast<AtomRec*>(ws + o_rec);
    float* pos_stage[2] = {reinterpret_cast<float*>(ws + o_pos0), reinterpret_cast<float*>(ws + o_pos1)};
    const float* f_dev = traj->f;
    if (pos_host && N > 0) {
        XS_CUDA(cudaMemcpyAsync(ws + o_f, traj->f, (size_t)N * sizeof(float), cudaMemcpyHostToDevice, st));
        f_dev = reinterpret_cast<float*>(ws + o_f);
    }

    const int64_t n_chunks = (int64_t)chunks.size();
    if (pos_host && N > 0) {
        // the copy stream starts after everything already on the caller's stream
        XS_CUDA(cudaEventRecord(ctx->ev_consumed[0], st));
        XS_CUDA(cudaEventRecord(ctx->ev_consumed[1], st));
    }
    auto issue_copy = [&](int64_t c) -> xs_status {
        const int64_t t0 = chunks[(size_t)c].first, nf = chunks[(size_t)c].second;
        const int b = (int)(c & 1);
        XS_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_consumed[b], 0));
        XS_CUDA(cudaMemcpyAsync(pos_stage[b], traj->pos + (size_t)t0 * N * 3, (size_t)nf * pos_per_frame,
                                cudaMemcpyHostToDevice, ctx->copy_stream));
        XS_CUDA(cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
        return XS_OK;
    };
    if (pos_host && N > 0) {
        s = issue_copy(0);
        if (s != XS_OK) return s;
    }
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t t0 = chunks[(size_t)c].first, nf = chunks[(size_t)c].second;
        float* Ic = out_dev ? I_out + (size_t)t0 * P : reinterpret_cast<float*>(ws + o_I);
        float* Ac = amp_out ? (out_dev ? amp_out + (size_t)t0 * P * 2 : reinterpret_cast<float*>(ws + o_amp)) : nullptr;
        if (N == 0) {
            XS_CUDA(cudaMemsetAsync(Ic, 0, (size_t)nf * P * sizeof(float), st));
            if (Ac) XS_CUDA(cudaMemsetAsync(Ac, 0, (size_t)nf * P * 2 * sizeof(float), st));
        } else {
            const float* pos_c;
            if (pos_host) {
                const int b = (int)(c & 1);
                if (c + 1 < n_chunks) {
                    s = issue_copy(c + 1);
                    if (s != XS_OK) return s;
                }
                XS_CUDA(cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
                pos_c = pos_stage[b];
            } else {
                pos_c = traj->pos + (size_t)t0 * N * 3;
            }
            XS_CUDA(traced(ctx, "phase", st, [&] { return launch_phase(pos_c, f_dev, N, nf, n_pad, hm, popt, rec, ctx->d_err, st); }));
            if (pos_host) XS_CUDA(cudaEventRecord(ctx->ev_consumed[c & 1], st));
            if (use_tc) {
                float* Ih = half_axis >= 0 ? reinterpret_cast<float*>(ws + o_half) : Ic;
                float* Ah = half_axis >= 0 ? (Ac ? reinterpret_cast<float*>(ws + o_half_amp) : nullptr) : Ac;
                const TcTraj tr = tc_traj(rec, n_pad, nf, gc, Ih, Ah, tile_kind, 0, ctx->exact_tables);
                const TcSplit sp = split_of(nf);
                XS_CUDA(traced(ctx, "tc", st, [&] {
                    return launch_tc_single(tr, tc_pairs, sp, chunk_stages, prec == XS_PREC_SPLIT_BF16,
                                            reinterpret_cast<double*>(ws + o_part), ws + o_split, ctx->d_err,
                                            ctx->timeout_ns, st);
                }));
                XS_CUDA(traced(ctx, "split_finish", st,
                               [&] { return launch_tc_split_finish(tr, tc_pairs, sp, ws + o_split, st); }));
                if (half_axis >= 0)
                    XS_CUDA(traced(ctx, "friedel", st,
                                   [&] { return launch_friedel(Ih, Ah, nf, gh, g, half_axis, Ic, Ac, st); }));
            } else if (factored) {
                const FactoredPlan pc = plan_factored(n_pad, nf, g, ctx->num_sms);
                if (pc.partial_bytes > fplan.partial_bytes) return fail(XS_ERR_CUDA, "internal: partial plan grew");
                XS_CUDA(traced(ctx, "factored", st,
                               [&] { return launch_factored(rec, n_pad, nf, g, pc, ws + o_part, Ic, Ac, st); }));
            } else {
                DirectPlan pc = plan_direct(n_pad, nf, g, ctx->num_sms);
                if (pc.partial_bytes > dplan.partial_bytes) return fail(XS_ERR_CUDA, "internal: partial plan grew");
                XS_CUDA(traced(ctx, "direct", st, [&] { return launch_direct(rec, n_pad, nf, g, pc, ws + o_part, Ic, Ac, st); }));
            }
        }
        if (!out_dev) {
            XS_CUDA(cudaMemcpyAsync(I_out + (size_t)t0 * P, Ic, (size_t)nf * P * sizeof(float), cudaMemcpyDeviceToHost, st));
            if (amp_out)
                XS_CUDA(cudaMemcpyAsync(amp_out + (size_t)t0 * P * 2, Ac, (size_t)nf * P * 2 * sizeof(float),
                                        cudaMemcpyDeviceToHost, st));
            XS_CUDA(cudaStreamSynchronize(st));
        }
    }
    if (pos_host && N > 0) XS_CUDA(cudaStreamSynchronize(st));  // host buffers may be released on return
    return XS_OK;
}

xs_status xs_intensity(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, xs_precision prec,
                       float* I_out, float* amp_out, void* cuda_stream) {
    return intensity_impl(ctx, traj, grid, prec, I_out, amp_out, static_cast<cudaStream_t>(cuda_stream), 0);
}

// --------------------------------------------------------------------------
// the FFT-based method (Algorithm 2), a cross-check
// --------------------------------------------------------------------------

xs_status xs_intensity_fft(xs_context* ctx, const xs_traj* traj, int32_t n_grid, double eta, int32_t k_cut,
                           const xs_qgrid* grid, float* I_out, float* amp_out, void* cuda_stream) {
    if (!ctx || !traj || !I_out) return fail(XS_ERR_INVALID_ARG, "context, trajectory and I_out are required");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (n_grid < 8 || n_grid > 1024 || (n_grid & (n_grid - 1)) != 0)
        return fail(XS_ERR_INVALID_ARG, "n_grid must be a power of two in [8, 1024]");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(XS_ERR_INVALID_ARG, "eta must be finite and > 0");
    if (traj->n_atoms < 0 || traj->n_frames < 0) return fail(XS_ERR_INVALID_ARG, "negative atom or frame count");
    if (traj->pos_on_host) return fail(XS_ERR_INVALID_ARG, "the FFT path takes device positions");
    if (traj->n_atoms > 0 && traj->n_frames > 0 && (!traj->pos || !traj->f))
        return fail(XS_ERR_INVALID_ARG, "positions or form factors are NULL");
    const double* h = traj->box.h;
    if (h[1] != 0.0 || h[2] != 0.0 || h[3] != 0.0 || h[5] != 0.0 || h[6] != 0.0 || h[7] != 0.0 ||
        !(h[0] > 0.0) || !(h[4] > 0.0) || !(h[8] > 0.0))
        return fail(XS_ERR_UNSUPPORTED, "the FFT path takes an orthorhombic cell");
    const int half = n_grid / 2;
    if (grid->nx0 < -half || grid->nx0 + grid->nx > half || grid->ny0 < -half || grid->ny0 + grid->ny > half ||
        grid->nz0 < -half || grid->nz0 + grid->nz > half)
        return fail(XS_ERR_INVALID_ARG, "Miller indices outside [-n_grid/2, n_grid/2) of the FFT grid");
    const GridDesc g = to_desc(grid);
    const int64_t P = g.pixels(), T = traj->n_frames, N = traj->n_atoms;
    if (P == 0 || T == 0) return XS_OK;
    if (!is_device_ptr(I_out) || (amp_out && !is_device_ptr(amp_out)))
        return fail(XS_ERR_INVALID_ARG, "the FFT path writes device outputs");
    FftGrid fg;
    fg.n = n_grid;
    fg.inv_2eta2 = 1.0 / (2.0 * eta * eta);
    const double Ls[3] = {h[0], h[4], h[8]};
    for (int a = 0; a < 3; ++a) {
        fg.h[a] = Ls[a] / n_grid;
        // k <= 0: the smallest integer above 10 eta in grid steps (+-5 eta)
        fg.k[a] = k_cut > 0 ? k_cut : (int)std::floor(10.0 * eta / fg.h[a]) + 1;
        if (fg.k[a] > 64 || fg.k[a] > n_grid)
            return fail(XS_ERR_INVALID_ARG, "Gaussian cut-off of %d grid points above min(64, n_grid)", fg.k[a]);
    }
    // G_a(m) = sum_j w_j exp(-2 pi i m x_j / n) of the truncated Gaussian at the origin
    std::vector<double> G((size_t)3 * n_grid * 2);
    const double two_pi = 6.283185307179586476925286766559;
    for (int a = 0; a < 3; ++a) {
        const int64_t s0 = (int64_t)std::ceil(-0.5 * fg.k[a]);
        for (int m = 0; m < n_grid; ++m) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < fg.k[a]; ++j) {
                const int64_t idx = s0 + j;
                const double d = (double)idx * fg.h[a];
                const double w = std::exp(-d * d / (2.0 * eta * eta));
                const int64_t e = ((idx % n_grid) + n_grid) % n_grid;
                const double ang = -two_pi * (double)((m * e) % n_grid) / n_grid;
                re += w * std::cos(ang);
                im += w * std::sin(ang);
            }
            G[((size_t)a * n_grid + m) * 2] = re;
            G[((size_t)a * n_grid + m) * 2 + 1] = im;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<char> blob;
    const size_t o_G = push(blob, G.data(), G.size());
    void* d = nullptr;
    s = upload_const(ctx, "fft", blob, st, &d);
    if (s != XS_OK) return s;
    const double2* d_G = reinterpret_cast<const double2*>(static_cast<char*>(d) + o_G);
    s = ensure_ws(ctx, (size_t)n_grid * n_grid * n_grid * sizeof(double2) + 256);
    if (s != XS_OK) return s;
    double2* fgrid = static_cast<double2*>(ctx->ws);
    for (int64_t t = 0; t < T; ++t) {
        const float* pos_t = traj->pos + (size_t)t * N * 3;
        float* It = I_out + (size_t)t * P;
        float* At = amp_out ? amp_out + (size_t)t * P * 2 : nullptr;
        XS_CUDA(traced(ctx, "fft", st, [&] {
            return launch_fft_frame(pos_t, traj->f, N, fg, fgrid, g, d_G, It, At, ctx->d_err, st);
        }));
    }
    return XS_OK;
}

// --------------------------------------------------------------------------
// arbitrary lattice points, and the Ewald-sphere detector slice
// --------------------------------------------------------------------------

xs_status xs_ewald_points(const xs_box* box, const double* k_in, int32_t nx0, int32_t nx, int32_t ny0, int32_t ny,
                          int32_t* miller_out, uint8_t* valid_out) {
    if (!box || !k_in || (!miller_out && (int64_t)nx * ny > 0)) return fail(XS_ERR_INVALID_ARG, "missing argument");
    if (nx < 0 || ny < 0) return fail(XS_ERR_INVALID_ARG, "negative window");
    double hinv[9];
    if (!invert3(box->h, hinv)) return fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    const double two_pi = 6.283185307179586476925286766559;
    // q = Ht n with Ht = 2 pi h^-T: column c of Ht is 2 pi (row c of h^-1)
    double Ht[3][3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) Ht[a][c] = two_pi * hinv[c * 3 + a];
    const double k[3] = {k_in[0], k_in[1], k_in[2]};
    const double kn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    if (!(kn > 0.0) || !std::isfinite(kn)) return fail(XS_ERR_INVALID_ARG, "k_in must be finite and non-zero");
    const double d[3] = {Ht[0][2], Ht[1][2], Ht[2][2]};
    const double A = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    auto sphere_dist = [&](const double* q0, double nz) {
        double s2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double v = q0[a] + nz * d[a] + k[a];
            s2 += v * v;
        }
        return std::fabs(std::sqrt(s2) - kn);
    };
    int64_t p = 0;
    for (int32_t iy = 0; iy < ny; ++iy)
        for (int32_t ix = 0; ix < nx; ++ix, ++p) {
            const double n0 = (double)(nx0 + ix), n1 = (double)(ny0 + iy);
            double q0[3];
            for (int a = 0; a < 3; ++a) q0[a] = Ht[a][0] * n0 + Ht[a][1] * n1;
            // |q0 + n d + k|^2 = |k|^2:  A n^2 + B n + C = 0
            const double B = 2.0 * (q0[0] * d[0] + q0[1] * d[1] + q0[2] * d[2] + d[0] * k[0] + d[1] * k[1] + d[2] * k[2]);
            const double C = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + 2.0 * (q0[0] * k[0] + q0[1] * k[1] + q0[2] * k[2]);
            const double disc = B * B - 4.0 * A * C;
            int64_t nz = 0;
            const bool ok = disc >= 0.0;
            if (ok) {
                const double sq = std::sqrt(disc);
                const double r1 = (-B + sq) / (2.0 * A), r2 = (-B - sq) / (2.0 * A);
                const double root = std::fabs(r1) <= std::fabs(r2) ? r1 : r2;
                const double lo = std::floor(root), hi = std::ceil(root);
                const double dl = sphere_dist(q0, lo), dh = sphere_dist(q0, hi);
                nz = (int64_t)((dl < dh || (dl == dh && std::fabs(lo) <= std::fabs(hi))) ? lo : hi);
                if (nz < INT32_MIN || nz > INT32_MAX) return fail(XS_ERR_INVALID_ARG, "n_z out of the int32 range");
            }
            miller_out[3 * p] = nx0 + ix;
            miller_out[3 * p + 1] = ny0 + iy;
            miller_out[3 * p + 2] = ok ? (int32_t)nz : 0;
            if (valid_out) valid_out[p] = ok ? 1 : 0;
        }
    return XS_OK;
}

xs_status xs_intensity_points(xs_context* ctx, const xs_traj* traj, const int32_t* miller, int64_t P,
                              xs_precision prec, float* I_out, float* amp_out, void* cuda_stream) {
    if (!ctx || !traj || (P > 0 && (!miller || !I_out))) return fail(XS_ERR_INVALID_ARG, "missing argument");
    if (prec != XS_PREC_FP32_DIRECT && prec != XS_PREC_SPLIT_FP16 && prec != XS_PREC_SPLIT_BF16)
        return fail(XS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (P < 0 || P > INT32_MAX) return fail(XS_ERR_INVALID_ARG, "point count outside [0, 2^31)");
    if (traj->n_atoms < 0 || traj->n_frames < 0) return fail(XS_ERR_INVALID_ARG, "negative atom or frame count");
    if (traj->n_atoms > (int64_t)1 << 31) return fail(XS_ERR_INVALID_ARG, "more than 2^31 atoms");
    if (traj->pos_on_host) return fail(XS_ERR_INVALID_ARG, "the point path takes device positions");
    if (traj->n_atoms > 0 && traj->n_frames > 0 && (!traj->pos || !traj->f))
        return fail(XS_ERR_INVALID_ARG, "positions or form factors are NULL");
    double hinv[9];
    if (!invert3(traj->box.h, hinv)) return fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    const int64_t T = traj->n_frames, N = traj->n_atoms;
    if (P == 0 || T == 0) return XS_OK;
    if (!is_device_ptr(I_out) || (amp_out && !is_device_ptr(amp_out)))
        return fail(XS_ERR_INVALID_ARG, "the point path writes device outputs");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (N == 0) {
        XS_CUDA(cudaMemsetAsync(I_out, 0, (size_t)T * P * sizeof(float), st));
        if (amp_out) XS_CUDA(cudaMemsetAsync(amp_out, 0, (size_t)T * P * 2 * sizeof(float), st));
        return XS_OK;
    }
    const bool use_tc = prec != XS_PREC_FP32_DIRECT;
    const int64_t n_pad = round_up(N, 64);
    Mat3 hm;
    for (int i = 0; i < 9; ++i) hm.a[i] = hinv[i];
    PhaseOpts popt;
    popt.ortho = is_ortho(hinv);
    popt.need_z = false;
    for (int64_t p = 0; p < P; ++p)
        if (miller[3 * p + 2] != 0) popt.need_z = true;
    popt.perm_mul = use_tc ? coprime_stride(n_pad / kPermRun) : 1;

    // tensor cores: the points grouped by n_z plane, each plane's bounding box
    // tiled; only tiles that hold a point are computed
    struct Plane {
        int32_t z, x0, x1, y0, y1;
        int64_t off;  // offset of the plane's box in a frame of the temporary buffer
    };
    std::vector<Plane> planes;
    std::vector<int32_t> plane_of((size_t)P);
    int64_t per_frame = 0;
    if (use_tc) {
        std::map<int32_t, size_t> index;
        for (int64_t p = 0; p < P; ++p) {
            const int32_t x = miller[3 * p], y = miller[3 * p + 1], z = miller[3 * p + 2];
            auto it = index.find(z);
            if (it == index.end()) {
                it = index.emplace(z, planes.size()).first;
                planes.push_back(Plane{z, x, x, y, y, 0});
            }
            Plane& pl = planes[it->second];
            pl.x0 = std::min(pl.x0, x);
            pl.x1 = std::max(pl.x1, x);
            pl.y0 = std::min(pl.y0, y);
            pl.y1 = std::max(pl.y1, y);
            plane_of[(size_t)p] = (int32_t)it->second;
        }
        for (Plane& pl : planes) {
            pl.off = per_frame;
            per_frame += (int64_t)(pl.x1 - pl.x0 + 1) * (pl.y1 - pl.y0 + 1);
        }
    }
    // frames per chunk
    const size_t bytes_frame = (size_t)n_pad * sizeof(AtomRec) +
                               (size_t)per_frame * (sizeof(float) + (amp_out ? 2 * sizeof(float) : 0));
    int64_t fchunk = std::max<int64_t>(1, std::min<int64_t>(T, (int64_t)(((size_t)4 << 30) / bytes_frame)));
    if (fchunk > 65535) fchunk = 65535;
    const GridDesc gpts{0, (int32_t)P, 0, 1, 0, 1};
    int tc_pairs = 0;
    DirectPlan dplan{};
    if (use_tc)
        tc_pairs = tc_pair_capacity(ctx->num_sms);
    else
        dplan = plan_direct(n_pad, fchunk, gpts, ctx->num_sms);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = round_up((int64_t)off, 256);
        off = o + bytes;
        return o;
    };
    const size_t o_rec = carve((size_t)fchunk * n_pad * sizeof(AtomRec));
    const size_t o_part = carve(use_tc ? tc_scratch_bytes(tc_pairs) : dplan.partial_bytes);
    const size_t o_tmp = carve(use_tc ? (size_t)fchunk * per_frame * sizeof(float) : 0);
    const size_t o_tamp = carve(use_tc && amp_out ? (size_t)fchunk * per_frame * 2 * sizeof(float) : 0);
    xs_status s = ensure_ws(ctx, off + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    AtomRec* rec = reinterpret_cast<AtomRec*>(ws + o_rec);

    for (int64_t t0 = 0; t0 < T; t0 += fchunk) {
        const int64_t nf = std::min(fchunk, T - t0);
        const float* pos_c = traj->pos + (size_t)t0 * N * 3;
        XS_CUDA(traced(ctx, "phase", st,
                       [&] { return launch_phase(pos_c, traj->f, N, nf, n_pad, hm, popt, rec, ctx->d_err, st); }));
        float* Ic = I_out + (size_t)t0 * P;
        float* Ac = amp_out ? amp_out + (size_t)t0 * P * 2 : nullptr;
        if (!use_tc) {
            std::vector<char> blob;
            const size_t o_pts = push(blob, miller, (size_t)P * 3);
            void* d = nullptr;
            s = upload_const(ctx, "points", blob, st, &d);
            if (s != XS_OK) return s;
            const int32_t* d_pts = reinterpret_cast<const int32_t*>(static_cast<char*>(d) + o_pts);
            const DirectPlan pc = plan_direct(n_pad, nf, gpts, ctx->num_sms);
            XS_CUDA(traced(ctx, "direct", st,
                           [&] { return launch_direct(rec, n_pad, nf, gpts, pc, ws + o_part, Ic, Ac, st, d_pts); }));
            continue;
        }
        float* tmp = reinterpret_cast<float*>(ws + o_tmp);
        float* tamp = amp_out ? reinterpret_cast<float*>(ws + o_tamp) : nullptr;
        std::vector<TcTraj> trs;
        for (const Plane& pl : planes) {
            GridDesc g{pl.x0, pl.x1 - pl.x0 + 1, pl.y0, pl.y1 - pl.y0 + 1, pl.z, 1};
            TcTraj tr = tc_traj(rec, n_pad, nf, g, nullptr, nullptr, kTcTile128, 0, ctx->exact_tables);
            // each plane writes its own [nf][box] block of the temporary buffer
            tr.I = tmp + (size_t)nf * pl.off;
            tr.amp = tamp ? tamp + (size_t)nf * pl.off * 2 : nullptr;
            trs.push_back(tr);
        }
        // occupied tiles, once per frame
        std::vector<int4> occupied;
        {
            std::vector<std::vector<uint8_t>> used(planes.size());
            for (size_t i = 0; i < planes.size(); ++i) used[i].assign((size_t)trs[i].tiles_x * trs[i].tiles_y, 0);
            for (int64_t p = 0; p < P; ++p) {
                const size_t i = (size_t)plane_of[(size_t)p];
                const int tx = (miller[3 * p] - planes[i].x0) / 128, ty = (miller[3 * p + 1] - planes[i].y0) / 128;
                used[i][(size_t)ty * trs[i].tiles_x + tx] = 1;
            }
            for (int64_t f = 0; f < nf; ++f)
                for (size_t i = 0; i < planes.size(); ++i)
                    for (int ty = 0; ty < trs[i].tiles_y; ++ty)
                        for (int tx = 0; tx < trs[i].tiles_x; ++tx)
                            if (used[i][(size_t)ty * trs[i].tiles_x + tx])
                                occupied.push_back(make_int4((int)i, (int)f, 0, tx | (ty << 16)));
        }
        const int n_pairs = (int)std::min<int64_t>(tc_pairs, (int64_t)occupied.size());
        std::vector<int4> units;
        std::vector<int> pair_start;
        tc_deal_units(trs, occupied, n_pairs, units, pair_start);
        // gather map: frame-0 offset and frame stride of every point
        std::vector<int64_t> src((size_t)P), stride((size_t)P);
        for (int64_t p = 0; p < P; ++p) {
            const Plane& pl = planes[(size_t)plane_of[(size_t)p]];
            const int64_t w = pl.x1 - pl.x0 + 1, area = w * (pl.y1 - pl.y0 + 1);
            src[(size_t)p] = nf * pl.off + (int64_t)(miller[3 * p + 1] - pl.y0) * w + (miller[3 * p] - pl.x0);
            stride[(size_t)p] = area;
        }
        std::vector<char> blob;
        const size_t o_tr = push(blob, trs.data(), trs.size());
        const size_t o_units = push(blob, units.data(), units.size());
        const size_t o_ps = push(blob, pair_start.data(), pair_start.size());
        const size_t o_src = push(blob, src.data(), src.size());
        const size_t o_stride = push(blob, stride.data(), stride.size());
        void* d = nullptr;
        s = upload_const(ctx, "points_tc", blob, st, &d);
        if (s != XS_OK) return s;
        char* dc = static_cast<char*>(d);
        XS_CUDA(traced(ctx, "tc", st, [&] {
            return launch_tc_batch(reinterpret_cast<const TcTraj*>(dc + o_tr), reinterpret_cast<const int4*>(dc + o_units),
                                   reinterpret_cast<const int*>(dc + o_ps), n_pairs, kDefaultChunkStages, prec == XS_PREC_SPLIT_BF16,
                                   kTcTile128, ctx->exact_tables,
                                   reinterpret_cast<double*>(ws + o_part), ctx->d_err, ctx->timeout_ns, st);
        }));
        XS_CUDA(traced(ctx, "points", st, [&] {
            return launch_points_gather(tmp, tamp, reinterpret_cast<const int64_t*>(dc + o_src),
                                        reinterpret_cast<const int64_t*>(dc + o_stride), P, nf, Ic, Ac, st);
        }));
    }
    return XS_OK;
}

// --------------------------------------------------------------------------
// several species with q-dependent form factors
// --------------------------------------------------------------------------

xs_status xs_intensity_species(xs_context* ctx, const xs_traj* traj, const int32_t* species, int32_t n_species,
                               const double* coef, const xs_qgrid* grid, xs_precision prec, float* I_out,
                               float* amp_out, void* cuda_stream) {
    if (!ctx || !traj || !I_out) return fail(XS_ERR_INVALID_ARG, "context, trajectory and I_out are required");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (prec != XS_PREC_FP32_DIRECT && prec != XS_PREC_SPLIT_FP16 && prec != XS_PREC_SPLIT_BF16)
        return fail(XS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (n_species < 1 || !coef) return fail(XS_ERR_INVALID_ARG, "need n_species >= 1 and the form factor table");
    for (int64_t i = 0; i < (int64_t)n_species * 9; ++i)
        if (!std::isfinite(coef[i])) return fail(XS_ERR_INVALID_ARG, "non-finite form factor coefficient");
    if (traj->n_atoms < 0 || traj->n_frames < 0) return fail(XS_ERR_INVALID_ARG, "negative atom or frame count");
    if (traj->n_atoms > (int64_t)1 << 31) return fail(XS_ERR_INVALID_ARG, "more than 2^31 atoms");
    if (traj->n_atoms > 0 && traj->n_frames > 0 && (!traj->pos || !traj->f || !species))
        return fail(XS_ERR_INVALID_ARG, "positions, weights or species are NULL");
    if (traj->pos_on_host) return fail(XS_ERR_INVALID_ARG, "the species path takes device positions");
    double hinv[9];
    if (!invert3(traj->box.h, hinv)) return fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    const GridDesc g = to_desc(grid);
    const int64_t P = g.pixels(), T = traj->n_frames, N = traj->n_atoms;
    if (P == 0 || T == 0) return XS_OK;
    if (!is_device_ptr(I_out) || (amp_out && !is_device_ptr(amp_out)))
        return fail(XS_ERR_INVALID_ARG, "the species path writes device outputs");
    if (N > 0 && !is_device_ptr(traj->pos)) return fail(XS_ERR_INVALID_ARG, "positions must be in device memory");
    const bool use_tc = prec != XS_PREC_FP32_DIRECT;
    if (use_tc && !tc_supported(g)) return fail(XS_ERR_UNSUPPORTED, "grid not supported by the tensor-core path");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // atoms grouped by species (stable)
    std::vector<int64_t> start((size_t)n_species + 1, 0);
    for (int64_t j = 0; j < N; ++j) {
        if (species[j] < 0 || species[j] >= n_species)
            return fail(XS_ERR_INVALID_ARG, "atom %lld has species %d outside [0, %d)", (long long)j, species[j], n_species);
        ++start[(size_t)species[j] + 1];
    }
    for (int sp = 0; sp < n_species; ++sp) start[(size_t)sp + 1] += start[(size_t)sp];
    std::vector<int32_t> index((size_t)std::max<int64_t>(N, 1), 0);
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t j = 0; j < N; ++j) index[(size_t)fill[(size_t)species[j]]++] = (int32_t)j;
    }
    int64_t n_pad_max = 64;
    for (int sp = 0; sp < n_species; ++sp)
        n_pad_max = std::max<int64_t>(n_pad_max, round_up(start[(size_t)sp + 1] - start[(size_t)sp], 64));
    std::vector<char> blob;
    const size_t o_coef = push(blob, coef, (size_t)n_species * 9);
    const size_t o_index = push(blob, index.data(), index.size());
    void* d = nullptr;
    s = upload_const(ctx, "species", blob, st, &d);
    if (s != XS_OK) return s;
    const double* d_coef = reinterpret_cast<const double*>(static_cast<char*>(d) + o_coef);
    const int32_t* d_index = reinterpret_cast<const int32_t*>(static_cast<char*>(d) + o_index);

    // frames per chunk: records plus the per-frame amplitude buffers
    const size_t per_frame = (size_t)n_pad_max * sizeof(AtomRec) + (size_t)P * (2 * sizeof(float) + sizeof(float) + 2 * sizeof(double));
    int64_t fchunk = std::max<int64_t>(1, std::min<int64_t>(T, (int64_t)(((size_t)6 << 30) / per_frame)));
    if (fchunk > 65535) fchunk = 65535;
    // tile kind and chunk length per species' atom count, as xs_intensity
    // chooses them (tuned per shape bucket, else the default rule)
    auto choice_of = [&](int64_t n_pad) {
        xs_context::TcChoice c{tc_default_kind(g), kDefaultChunkStages};
        auto it = ctx->tuned.find(tc_bucket(n_pad, g, (int)prec));
        if (it != ctx->tuned.end()) c = it->second;
        return c;
    };
    int tc_pairs = 0;
    DirectPlan dmax{};
    if (use_tc) {
        tc_pairs = std::max(tc_pair_capacity(ctx->num_sms, kTcTile128), tc_pair_capacity(ctx->num_sms, kTcTile64));
    } else {
        for (int sp = 0; sp < n_species; ++sp) {
            const int64_t n = start[(size_t)sp + 1] - start[(size_t)sp];
            if (n == 0) continue;
            const DirectPlan pl = plan_direct(round_up(n, 64), fchunk, g, ctx->num_sms);
            if (pl.partial_bytes > dmax.partial_bytes) dmax = pl;
        }
    }
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = round_up((int64_t)off, 256);
        off = o + bytes;
        return o;
    };
    const size_t o_rec = carve((size_t)fchunk * n_pad_max * sizeof(AtomRec));
    const size_t o_part = carve(use_tc ? tc_scratch_bytes(tc_pairs) : dmax.partial_bytes);
    auto split_of = [&](int64_t n_pad, int64_t nf) {
        const xs_context::TcChoice c = choice_of(n_pad);
        return tc_split_plan(tc_units(tc_traj(nullptr, n_pad, nf, g, nullptr, nullptr, c.kind)),
                             tc_pair_capacity(ctx->num_sms, c.kind), (int)(n_pad / tc_atom_multiple()), c.chunk);
    };
    size_t split_bytes = 0;
    if (use_tc) {
        for (int sp = 0; sp < n_species; ++sp) {
            const int64_t ns = start[(size_t)sp + 1] - start[(size_t)sp];
            if (ns == 0) continue;
            split_bytes = std::max(split_bytes, tc_split_bytes(split_of(round_up(ns, 64), fchunk)));
            split_bytes = std::max(split_bytes, tc_split_bytes(split_of(round_up(ns, 64), T - (T - 1) / fchunk * fchunk)));
        }
    }
    const size_t o_split = carve(split_bytes);
    const size_t o_S = carve((size_t)fchunk * P * 2 * sizeof(float));
    const size_t o_I = carve((size_t)fchunk * P * sizeof(float));
    const size_t o_acc = carve((size_t)fchunk * P * 2 * sizeof(double));
    const size_t o_ff = carve((size_t)n_species * P * sizeof(double));
    s = ensure_ws(ctx, off + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    AtomRec* rec = reinterpret_cast<AtomRec*>(ws + o_rec);
    float* S_tmp = reinterpret_cast<float*>(ws + o_S);
    float* I_tmp = reinterpret_cast<float*>(ws + o_I);
    double* acc = reinterpret_cast<double*>(ws + o_acc);
    double* ff = reinterpret_cast<double*>(ws + o_ff);
    Mat3 hm;
    for (int i = 0; i < 9; ++i) hm.a[i] = hinv[i];
    XS_CUDA(traced(ctx, "species", st, [&] { return launch_ff_table(d_coef, n_species, g, hm, ff, st); }));

    for (int64_t t0 = 0; t0 < T; t0 += fchunk) {
        const int64_t nf = std::min(fchunk, T - t0);
        bool first = true;
        for (int sp = 0; sp < n_species; ++sp) {
            const int64_t ns = start[(size_t)sp + 1] - start[(size_t)sp];
            if (ns == 0) continue;
            const int64_t n_pad = round_up(ns, 64);
            PhaseOpts popt;
            popt.ortho = is_ortho(hinv);
            popt.need_z = !(g.nz == 1 && g.nz0 == 0);
            popt.perm_mul = use_tc ? coprime_stride(n_pad / kPermRun) : 1;
            popt.index = d_index + start[(size_t)sp];
            popt.pos_atoms = N;
            const float* pos_c = traj->pos + (size_t)t0 * N * 3;
            XS_CUDA(traced(ctx, "phase", st,
                           [&] { return launch_phase(pos_c, traj->f, ns, nf, n_pad, hm, popt, rec, ctx->d_err, st); }));
            if (use_tc) {
                const xs_context::TcChoice ch = choice_of(n_pad);
                const int pairs = tc_pair_capacity(ctx->num_sms, ch.kind);
                const TcTraj tr = tc_traj(rec, n_pad, nf, g, I_tmp, S_tmp, ch.kind, 0, ctx->exact_tables);
                const TcSplit spl = split_of(n_pad, nf);
                XS_CUDA(traced(ctx, "tc", st, [&] {
                    return launch_tc_single(tr, pairs, spl, ch.chunk, prec == XS_PREC_SPLIT_BF16,
                                            reinterpret_cast<double*>(ws + o_part), ws + o_split, ctx->d_err,
                                            ctx->timeout_ns, st);
                }));
                XS_CUDA(traced(ctx, "split_finish", st,
                               [&] { return launch_tc_split_finish(tr, pairs, spl, ws + o_split, st); }));
            } else {
                const DirectPlan pc = plan_direct(n_pad, nf, g, ctx->num_sms);
                if (pc.partial_bytes > dmax.partial_bytes) return fail(XS_ERR_CUDA, "internal: partial plan grew");
                XS_CUDA(traced(ctx, "direct", st,
                               [&] { return launch_direct(rec, n_pad, nf, g, pc, ws + o_part, I_tmp, S_tmp, st); }));
            }
            XS_CUDA(traced(ctx, "species", st, [&] {
                return launch_species_acc(S_tmp, ff + (size_t)sp * P, nf, P, first, acc, st);
            }));
            first = false;
        }
        float* Ic = I_out + (size_t)t0 * P;
        float* Ac = amp_out ? amp_out + (size_t)t0 * P * 2 : nullptr;
        if (first) {  // no atoms at all
            XS_CUDA(cudaMemsetAsync(Ic, 0, (size_t)nf * P * sizeof(float), st));
            if (Ac) XS_CUDA(cudaMemsetAsync(Ac, 0, (size_t)nf * P * 2 * sizeof(float), st));
        } else {
            XS_CUDA(traced(ctx, "species", st, [&] { return launch_species_finish(acc, nf * P, Ic, Ac, st); }));
        }
    }
    return XS_OK;
}

xs_status xs_tune(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, xs_precision prec, void* cuda_stream) {
    if (!ctx || !traj || !grid) return fail(XS_ERR_INVALID_ARG, "bad tune arguments");
    if (prec == XS_PREC_FP32_DIRECT || prec == XS_PREC_FP32_FACTORED) return XS_OK;
    if (traj->pos_on_host) return fail(XS_ERR_INVALID_ARG, "tuning needs device positions");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const GridDesc g = to_desc(grid);
    const int64_t P = g.pixels();
    const int64_t T = std::min<int64_t>(traj->n_frames, 64);
    if (P == 0 || T == 0 || traj->n_atoms == 0) return XS_OK;
    // the grid the contraction runs on (a half grid where that saves tiles,
    // always on 128 x 128 tiles) and the key the intensity calls look up
    GridDesc gc = g;
    const bool half = friedel_half_grid(g, gc) >= 0;
    if (!half) gc = g;
    const int64_t n_pad = round_up(traj->n_atoms, 64);
    XS_CUDA(cudaStreamSynchronize(st));
    float* out = static_cast<float*>(ctx->raw_alloc((size_t)T * P * sizeof(float)));
    if (!out) return fail(XS_ERR_NO_MEMORY, "tuning buffer allocation failed");
    xs_traj sub = *traj;
    sub.n_frames = T;
    cudaEvent_t e0, e1;
    XS_CUDA(cudaEventCreate(&e0));
    XS_CUDA(cudaEventCreate(&e1));
    // tile kinds x chunk lengths, each timed as the fastest of three calls
    // after a warm-up call.  The untuned choice is timed first and is kept
    // unless another one is faster by more than 1%, so that timing noise
    // does not replace it by an equal or slower one.  The tensor core's FP32
    // accumulation is not round-to-nearest: no chunk longer than 4,096 atoms,
    // so its bias stays far below the 1e-4 target
    const xs_context::TcChoice dflt{half ? kTcTile128 : tc_default_kind(gc), kDefaultChunkStages};
    std::vector<xs_context::TcChoice> cands = {dflt};
    for (int kind : {kTcTile128, kTcTile64}) {
        if (half && kind != kTcTile128) continue;
        for (int c : {16, 32, 64})
            if (kind != dflt.kind || c != dflt.chunk) cands.push_back({kind, c});
    }
    xs_context::TcChoice best = dflt;
    float best_ms = 1e30f;
    for (size_t i = 0; i < cands.size() && s == XS_OK; ++i) {
        const xs_context::TcChoice cand = cands[i];
        s = intensity_impl(ctx, &sub, grid, prec, out, nullptr, st, cand.chunk, cand.kind);  // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && s == XS_OK; ++rep) {
            XS_CUDA(cudaEventRecord(e0, st));
            s = intensity_impl(ctx, &sub, grid, prec, out, nullptr, st, cand.chunk, cand.kind);
            if (s != XS_OK) break;
            XS_CUDA(cudaEventRecord(e1, st));
            XS_CUDA(cudaEventSynchronize(e1));
            float r = 0.f;
            XS_CUDA(cudaEventElapsedTime(&r, e0, e1));
            ms = std::min(ms, r);
        }
        if (s == XS_OK && (i == 0 || ms < 0.99f * best_ms)) {
            best_ms = ms;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    ctx->raw_free(out);
    if (s != XS_OK) return s;
    ctx->tuned[tc_bucket(n_pad, gc, (int)prec)] = best;
    return xs_sync_status(ctx, cuda_stream);
}

xs_status xs_tuned_choice(xs_context* ctx, int64_t n_atoms, const xs_qgrid* grid, xs_precision prec,
                          int32_t* tile_kind, int32_t* chunk_stages) {
    if (!ctx || !grid || !tile_kind || !chunk_stages || n_atoms < 0) return fail(XS_ERR_INVALID_ARG, "bad arguments");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    const GridDesc g = to_desc(grid);
    GridDesc gc = g;
    const bool half = friedel_half_grid(g, gc) >= 0;
    if (!half) gc = g;
    const int64_t n_pad = round_up(n_atoms > 0 ? n_atoms : 1, 64);
    auto it = ctx->tuned.find(tc_bucket(n_pad, gc, (int)prec));
    if (it == ctx->tuned.end()) {
        *tile_kind = half ? kTcTile128 : tc_default_kind(gc);
        *chunk_stages = kDefaultChunkStages;
        return XS_OK;
    }
    *tile_kind = half ? kTcTile128 : it->second.kind;
    *chunk_stages = it->second.chunk;
    return XS_OK;
}

// --------------------------------------------------------------------------
// g2
// --------------------------------------------------------------------------

xs_status xs_g2(xs_context* ctx, const float* I, int64_t T, int64_t P, const int32_t* taus, int32_t n_tau,
                double* g2_out, double* mean_out, void* cuda_stream) {
    if (!ctx || !I || !taus || !g2_out) return fail(XS_ERR_INVALID_ARG, "context, I, taus and g2_out are required");
    if (T < 1 || P < 0 || n_tau < 0) return fail(XS_ERR_INVALID_ARG, "need T >= 1, P >= 0, n_tau >= 0");
    for (int32_t k = 0; k < n_tau; ++k)
        if (taus[k] < 0 || taus[k] >= T) return fail(XS_ERR_INVALID_ARG, "delay %d outside [0, T)", taus[k]);
    if (P == 0 || n_tau == 0) return XS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<char> blob;
    const size_t o_tau = push(blob, taus, (size_t)n_tau);
    void* d = nullptr;
    xs_status s = upload_const(ctx, "g2", blob, st, &d);
    if (s != XS_OK) return s;
    const int32_t* d_taus = reinterpret_cast<const int32_t*>(static_cast<char*>(d) + o_tau);
    s = ensure_ws(ctx, g2_workspace_bytes(T, P, n_tau) + 256);
    if (s != XS_OK) return s;
    void* ws = ctx->ws;
    XS_CUDA(traced(ctx, "g2", st, [&] { return launch_g2(I, T, P, d_taus, n_tau, g2_out, mean_out, ws, st); }));
    return XS_OK;
}

// --------------------------------------------------------------------------
// XSVS contrast
// --------------------------------------------------------------------------

// ring (1..n_rings) of each pixel, 0 when in none; shared by the contrast call
// and the host-side layout export below
static xs_status ring_of_pixels(const xs_qgrid* grid, const xs_box* box, double ring_width, int32_t n_rings,
                                std::vector<int32_t>& ring) {
    double hinv[9];
    if (!invert3(box->h, hinv)) return fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    const double* h = box->h;
    const double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                       h[2] * (h[3] * h[7] - h[4] * h[6]);
    const double two_pi = 6.283185307179586476925286766559;
    const double delta = two_pi / std::cbrt(std::fabs(det));
    const int64_t P = (int64_t)grid->nx * grid->ny * grid->nz;
    ring.assign((size_t)P, 0);
    int64_t p = 0;
    for (int iz = 0; iz < grid->nz; ++iz)
        for (int iy = 0; iy < grid->ny; ++iy)
            for (int ix = 0; ix < grid->nx; ++ix, ++p) {
                const double n[3] = {(double)(grid->nx0 + ix), (double)(grid->ny0 + iy), (double)(grid->nz0 + iz)};
                double q2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double qa = two_pi * (hinv[0 * 3 + a] * n[0] + hinv[1 * 3 + a] * n[1] + hinv[2 * 3 + a] * n[2]);
                    q2 += qa * qa;
                }
                const double x = std::sqrt(q2) / delta;
                const double r = std::floor(x + 0.5);
                if (r >= 1.0 && r <= (double)n_rings && x >= r - ring_width / 2.0 && x < r + ring_width / 2.0)
                    ring[(size_t)p] = (int32_t)r;
            }
    return XS_OK;
}

xs_status xs_ring_index(const xs_qgrid* grid, const xs_box* box, double ring_width, int32_t n_rings,
                        int32_t* ring_out) {
    if (!grid || !box || !ring_out) return fail(XS_ERR_INVALID_ARG, "grid, box and ring_out are required");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (!(ring_width > 0.0 && ring_width <= 1.0) || n_rings < 0) return fail(XS_ERR_INVALID_ARG, "bad ring parameters");
    std::vector<int32_t> ring;
    s = ring_of_pixels(grid, box, ring_width, n_rings, ring);
    if (s != XS_OK) return s;
    if (!ring.empty()) std::memcpy(ring_out, ring.data(), ring.size() * sizeof(int32_t));
    return XS_OK;
}

// pixels grouped ring by ring (stable within a ring): perm[start[r] ..
// start[r+1]) are the pixels of ring r + 1
struct RingLayout {
    std::vector<int32_t> count;
    std::vector<int64_t> start;
    std::vector<int32_t> perm;
};

static xs_status ring_layout(const xs_qgrid* grid, const xs_box* box, double ring_width, int32_t n_rings,
                             RingLayout& out) {
    std::vector<int32_t> ring;
    xs_status s = ring_of_pixels(grid, box, ring_width, n_rings, ring);
    if (s != XS_OK) return s;
    const int64_t P = (int64_t)ring.size();
    out.count.assign((size_t)n_rings, 0);
    for (int32_t r : ring)
        if (r > 0) ++out.count[(size_t)r - 1];
    out.start.assign((size_t)n_rings + 1, 0);
    for (int r = 0; r < n_rings; ++r) out.start[(size_t)r + 1] = out.start[(size_t)r] + out.count[(size_t)r];
    out.perm.assign((size_t)out.start[(size_t)n_rings], 0);
    std::vector<int64_t> fill(out.start.begin(), out.start.end() - 1);
    for (int64_t p = 0; p < P; ++p)
        if (ring[(size_t)p] > 0) out.perm[(size_t)fill[(size_t)ring[(size_t)p] - 1]++] = (int32_t)p;
    return XS_OK;
}

// Host tables of the XSVS contrast of one grid (Eqs. inte_Iq, bq_Iq): pixels
// grouped by ring, (ring, start, count) chunks of at most 128 pixels, the
// first chunk of each ring, and the offset of each window length's windows in
// the (K, w) list.
struct XsvsTables {
    std::vector<int32_t> count, perm, chunks, first;
    std::vector<int64_t> kw_off;
    int64_t n_in = 0, n_kw = 0;
    int n_chunks = 0;
};

static xs_status xsvs_tables(const xs_qgrid* grid, const xs_box* box, double ring_width, int32_t n_rings,
                             const int32_t* Ks, int32_t n_K, int64_t T, XsvsTables& t) {
    RingLayout lay;
    xs_status s = ring_layout(grid, box, ring_width, n_rings, lay);
    if (s != XS_OK) return s;
    t.count = std::move(lay.count);
    t.perm = std::move(lay.perm);
    t.n_in = lay.start[(size_t)n_rings];
    constexpr int kChunk = 128;
    t.chunks.clear();  // int4 records (ring, start, count, 0)
    t.first.assign((size_t)n_rings + 1, 0);
    for (int r = 0; r < n_rings; ++r) {
        t.first[(size_t)r] = (int32_t)(t.chunks.size() / 4);
        for (int64_t a = lay.start[(size_t)r]; a < lay.start[(size_t)r + 1]; a += kChunk) {
            t.chunks.push_back(r + 1);
            t.chunks.push_back((int32_t)a);
            t.chunks.push_back((int32_t)std::min<int64_t>(kChunk, lay.start[(size_t)r + 1] - a));
            t.chunks.push_back(0);
        }
    }
    t.n_chunks = (int)(t.chunks.size() / 4);
    t.first[(size_t)n_rings] = t.n_chunks;
    t.kw_off.assign((size_t)n_K + 1, 0);
    for (int k = 0; k < n_K; ++k) t.kw_off[(size_t)k + 1] = t.kw_off[(size_t)k] + T / Ks[k];
    t.n_kw = t.kw_off[(size_t)n_K];
    return XS_OK;
}

// workspace of one XSVS evaluation: FP64 prefix rows, then (K, w) partials
static size_t xsvs_prefix_bytes(int64_t T, const XsvsTables& t) {
    return (size_t)round_up((int64_t)((size_t)xsvs_prefix_rows(T) * t.n_in * sizeof(double)), 256);
}
static size_t xsvs_ws_bytes(int64_t T, const XsvsTables& t) {
    return xsvs_prefix_bytes(T, t) + (size_t)t.n_kw * t.n_chunks * sizeof(double2);
}

// --------------------------------------------------------------------------
// XSVS over pixel shards: partial sums on the device, finalize on the host
// --------------------------------------------------------------------------

xs_status xs_xsvs_partial(xs_context* ctx, const float* I, int64_t T, int64_t P, const int32_t* ring, int32_t n_rings,
                          const int32_t* Ks, int32_t n_K, double* sums_out, int64_t* count_out, void* cuda_stream) {
    if (!ctx || (P > 0 && (!I || !ring)) || (n_K > 0 && !Ks)) return fail(XS_ERR_INVALID_ARG, "missing argument");
    if (T < 1 || P < 0 || n_K < 0 || n_rings < 0) return fail(XS_ERR_INVALID_ARG, "need T >= 1, P, n_K, n_rings >= 0");
    if (P > INT32_MAX) return fail(XS_ERR_INVALID_ARG, "more than 2^31 pixels");
    for (int32_t k = 0; k < n_K; ++k)
        if (Ks[k] < 1 || Ks[k] > T) return fail(XS_ERR_INVALID_ARG, "window length %d outside [1, T]", Ks[k]);
    std::vector<int32_t> count((size_t)n_rings, 0);
    for (int64_t p = 0; p < P; ++p) {
        if (ring[p] < 0 || ring[p] > n_rings) return fail(XS_ERR_INVALID_ARG, "pixel %lld has ring %d", (long long)p, ring[p]);
        if (ring[p] > 0) ++count[(size_t)ring[p] - 1];
    }
    if (count_out)
        for (int r = 0; r < n_rings; ++r) count_out[r] = count[(size_t)r];
    std::vector<int64_t> kw_off((size_t)n_K + 1, 0);
    for (int k = 0; k < n_K; ++k) kw_off[(size_t)k + 1] = kw_off[(size_t)k] + T / Ks[k];
    const int64_t n_kw = kw_off[(size_t)n_K];
    if (n_kw == 0 || n_rings == 0) return XS_OK;
    if (!sums_out) return fail(XS_ERR_INVALID_ARG, "sums_out is required");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<int64_t> start((size_t)n_rings + 1, 0);
    for (int r = 0; r < n_rings; ++r) start[(size_t)r + 1] = start[(size_t)r] + count[(size_t)r];
    const int64_t n_in = start[(size_t)n_rings];
    std::vector<int32_t> perm((size_t)std::max<int64_t>(n_in, 1), 0);
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t p = 0; p < P; ++p)
            if (ring[p] > 0) perm[(size_t)fill[(size_t)ring[p] - 1]++] = (int32_t)p;
    }
    constexpr int kChunk = 128;
    std::vector<int32_t> chunks, first((size_t)n_rings + 1, 0);
    for (int r = 0; r < n_rings; ++r) {
        first[(size_t)r] = (int32_t)(chunks.size() / 4);
        for (int64_t a = start[(size_t)r]; a < start[(size_t)r + 1]; a += kChunk) {
            chunks.push_back(r + 1);
            chunks.push_back((int32_t)a);
            chunks.push_back((int32_t)std::min<int64_t>(kChunk, start[(size_t)r + 1] - a));
            chunks.push_back(0);
        }
    }
    const int n_chunks = (int)(chunks.size() / 4);
    first[(size_t)n_rings] = n_chunks;
    if (chunks.empty()) chunks.assign(4, 0);
    std::vector<char> blob;
    const int64_t key[2] = {T, P};
    push(blob, key, 2);
    const size_t o_perm = push(blob, perm.data(), perm.size());
    const size_t o_chunks = push(blob, chunks.data(), chunks.size());
    const size_t o_K = push(blob, Ks, (size_t)n_K);
    const size_t o_kw = push(blob, kw_off.data(), kw_off.size());
    const size_t o_first = push(blob, first.data(), first.size());
    void* d = nullptr;
    xs_status s = upload_const(ctx, "xsvs_partial", blob, st, &d);
    if (s != XS_OK) return s;
    char* dc = static_cast<char*>(d);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = round_up((int64_t)off, 256);
        off = o + bytes;
        return o;
    };
    const size_t o_prefix = carve((size_t)xsvs_prefix_rows(T) * std::max<int64_t>(n_in, 1) * sizeof(double));
    const size_t o_partial = carve((size_t)n_kw * std::max(n_chunks, 1) * sizeof(double2));
    s = ensure_ws(ctx, off + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    if (n_chunks == 0) {  // no pixel in any ring: zero sums
        XS_CUDA(cudaMemsetAsync(sums_out, 0, (size_t)n_kw * n_rings * 2 * sizeof(double), st));
        return XS_OK;
    }
    XS_CUDA(traced(ctx, "xsvs", st, [&] {
        return launch_xsvs_partial(I, T, P, reinterpret_cast<const int32_t*>(dc + o_perm),
                                   reinterpret_cast<const int4*>(dc + o_chunks), n_chunks, n_in,
                                   reinterpret_cast<const int32_t*>(dc + o_K), reinterpret_cast<const int64_t*>(dc + o_kw),
                                   n_K, n_kw, reinterpret_cast<const int32_t*>(dc + o_first), n_rings,
                                   reinterpret_cast<double*>(ws + o_prefix), reinterpret_cast<double2*>(ws + o_partial),
                                   sums_out, st);
    }));
    return XS_OK;
}

xs_status xs_xsvs_finalize(const double* sums, const int64_t* counts, int64_t T, const int32_t* Ks, int32_t n_K,
                           int32_t n_rings, double* beta_out) {
    if ((n_K > 0 && (!Ks || !beta_out)) || (n_rings > 0 && !counts) || T < 1 || n_K < 0 || n_rings < 0)
        return fail(XS_ERR_INVALID_ARG, "bad arguments");
    int64_t kw0 = 0;
    for (int32_t k = 0; k < n_K; ++k) {
        if (Ks[k] < 1 || Ks[k] > T) return fail(XS_ERR_INVALID_ARG, "window length %d outside [1, T]", Ks[k]);
        const int64_t W = T / Ks[k];
        if (W > 0 && n_rings > 0 && !sums) return fail(XS_ERR_INVALID_ARG, "sums are required");
        for (int32_t r = 0; r < n_rings; ++r) {
            const double n = (double)counts[r];
            double acc = 0.0;
            for (int64_t w = 0; w < W; ++w) {
                const double* v = sums + ((kw0 + w) * n_rings + r) * 2;
                const double m1 = v[0] / n, m2 = v[1] / n;
                acc += (m2 - m1 * m1) / (m1 * m1);
            }
            beta_out[(int64_t)k * n_rings + r] = counts[r] > 0 ? acc / (double)W : std::nan("");
        }
        kw0 += W;
    }
    return XS_OK;
}

xs_status xs_xsvs_contrast(xs_context* ctx, const float* I, int64_t T, const xs_qgrid* grid, const xs_box* box,
                           const int32_t* Ks, int32_t n_K, double ring_width, int32_t n_rings, double* beta_out,
                           int32_t* ring_count_out, void* cuda_stream) {
    if (!ctx || !I || !box || !Ks || !beta_out) return fail(XS_ERR_INVALID_ARG, "missing argument");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (T < 1 || n_K < 0 || n_rings < 0) return fail(XS_ERR_INVALID_ARG, "need T >= 1, n_K >= 0, n_rings >= 0");
    if (!(ring_width > 0.0 && ring_width <= 1.0)) return fail(XS_ERR_INVALID_ARG, "ring_width must be in (0, 1]");
    for (int32_t k = 0; k < n_K; ++k)
        if (Ks[k] < 1 || Ks[k] > T) return fail(XS_ERR_INVALID_ARG, "window length %d outside [1, T]", Ks[k]);
    if (n_K == 0 || n_rings == 0) return XS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    XsvsTables t;
    s = xsvs_tables(grid, box, ring_width, n_rings, Ks, n_K, T, t);
    if (s != XS_OK) return s;
    const int64_t P = (int64_t)grid->nx * grid->ny * grid->nz;
    if (ring_count_out) std::memcpy(ring_count_out, t.count.data(), t.count.size() * sizeof(int32_t));

    std::vector<char> blob;
    const int64_t key[2] = {T, P};
    push(blob, key, 2);
    const size_t o_perm = push(blob, t.perm.data(), t.perm.size());
    const size_t o_chunks = push(blob, t.chunks.data(), t.chunks.size());
    const size_t o_K = push(blob, Ks, (size_t)n_K);
    const size_t o_kw = push(blob, t.kw_off.data(), t.kw_off.size());
    const size_t o_first = push(blob, t.first.data(), t.first.size());
    const size_t o_count = push(blob, t.count.data(), t.count.size());
    void* d = nullptr;
    s = upload_const(ctx, "xsvs", blob, st, &d);
    if (s != XS_OK) return s;
    char* dc = static_cast<char*>(d);
    s = ensure_ws(ctx, xsvs_ws_bytes(T, t) + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    const size_t o_prefix = 0, o_partial = xsvs_prefix_bytes(T, t);
    const int n_chunks = t.n_chunks;
    const int64_t n_in = t.n_in, n_kw = t.n_kw;
    XS_CUDA(traced(ctx, "xsvs", st, [&] { return launch_xsvs(I, T, P, reinterpret_cast<const int32_t*>(dc + o_perm), reinterpret_cast<const int4*>(dc + o_chunks),
                        n_chunks, n_in, reinterpret_cast<const int32_t*>(dc + o_K), reinterpret_cast<const int64_t*>(dc + o_kw),
                        n_K, n_kw, reinterpret_cast<const int32_t*>(dc + o_first), reinterpret_cast<const int32_t*>(dc + o_count),
                        n_rings, reinterpret_cast<double*>(ws + o_prefix), reinterpret_cast<double2*>(ws + o_partial),
                        beta_out, st); }));
    return XS_OK;
}

// --------------------------------------------------------------------------
// batched trajectories: intensities, then g2 and XSVS per trajectory
// --------------------------------------------------------------------------

// One trajectory's correlation stages in the batched pipeline: the delays and
// the XSVS tables live in the call's device blob at the recorded offsets.
struct CorrPrep {
    bool g2 = false, xsvs = false;
    int64_t T = 0, P = 0;
    int n_tau = 0;
    size_t o_taus = 0;
    XsvsTables t;
    int n_K = 0, n_rings = 0;
    size_t o_perm = 0, o_chunks = 0, o_K = 0, o_kw = 0, o_first = 0, o_count = 0;
    size_t ws_bytes = 0;
};

// Validates request `r` of a trajectory with T frames on `grid` and appends
// its device tables to `blob`.
static xs_status corr_prepare(const xs_corr_request& r, int32_t i, int64_t T, const xs_qgrid* grid,
                              const xs_box* box, std::vector<char>& blob, CorrPrep& cp) {
    const int64_t P = (int64_t)grid->nx * grid->ny * grid->nz;
    cp.T = T;
    cp.P = P;
    if (r.n_tau < 0 || r.n_K < 0 || r.n_rings < 0) return fail(XS_ERR_INVALID_ARG, "request %d: negative count", i);
    if (r.n_tau > 0) {
        if (!r.taus || !r.g2_out) return fail(XS_ERR_INVALID_ARG, "request %d: taus and g2_out are required", i);
        for (int32_t k = 0; k < r.n_tau; ++k)
            if (r.taus[k] < 0 || r.taus[k] >= T)
                return fail(XS_ERR_INVALID_ARG, "request %d: delay %d outside [0, %lld)", i, r.taus[k], (long long)T);
    }
    if (r.n_K > 0 && r.n_rings > 0) {
        if (!r.Ks || !r.beta_out) return fail(XS_ERR_INVALID_ARG, "request %d: Ks and beta_out are required", i);
        if (!(r.ring_width > 0.0 && r.ring_width <= 1.0))
            return fail(XS_ERR_INVALID_ARG, "request %d: ring_width must be in (0, 1]", i);
        for (int32_t k = 0; k < r.n_K; ++k)
            if (r.Ks[k] < 1 || r.Ks[k] > T)
                return fail(XS_ERR_INVALID_ARG, "request %d: window length %d outside [1, %lld]", i, r.Ks[k],
                            (long long)T);
    }
    if (P == 0 || T == 0) return XS_OK;
    if (r.n_tau > 0) {
        cp.g2 = true;
        cp.n_tau = r.n_tau;
        cp.o_taus = push(blob, r.taus, (size_t)r.n_tau);
        cp.ws_bytes = std::max(cp.ws_bytes, g2_workspace_bytes(T, P, r.n_tau));
    }
    if (r.n_K > 0 && r.n_rings > 0) {
        xs_status s = xsvs_tables(grid, box, r.ring_width, r.n_rings, r.Ks, r.n_K, T, cp.t);
        if (s != XS_OK) return s;
        if (r.ring_count_out) std::memcpy(r.ring_count_out, cp.t.count.data(), cp.t.count.size() * sizeof(int32_t));
        cp.xsvs = true;
        cp.n_K = r.n_K;
        cp.n_rings = r.n_rings;
        cp.o_perm = push(blob, cp.t.perm.data(), cp.t.perm.size());
        cp.o_chunks = push(blob, cp.t.chunks.data(), cp.t.chunks.size());
        cp.o_K = push(blob, r.Ks, (size_t)r.n_K);
        cp.o_kw = push(blob, cp.t.kw_off.data(), cp.t.kw_off.size());
        cp.o_first = push(blob, cp.t.first.data(), cp.t.first.size());
        cp.o_count = push(blob, cp.t.count.data(), cp.t.count.size());
        cp.ws_bytes = std::max(cp.ws_bytes, xsvs_ws_bytes(T, cp.t));
    }
    return XS_OK;
}

// Launches one trajectory's correlation stages (stream order: after its
// intensity); `dc` is the device copy of the blob, `cws` the shared workspace.
static cudaError_t corr_launch(const CorrPrep& cp, const xs_corr_request& r, const float* I, const char* dc,
                               char* cws, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (cp.g2)
        e = launch_g2(I, cp.T, cp.P, reinterpret_cast<const int32_t*>(dc + cp.o_taus), cp.n_tau, r.g2_out, r.mean_out,
                      cws, st);
    if (e == cudaSuccess && cp.xsvs)
        e = launch_xsvs(I, cp.T, cp.P, reinterpret_cast<const int32_t*>(dc + cp.o_perm),
                        reinterpret_cast<const int4*>(dc + cp.o_chunks), cp.t.n_chunks, cp.t.n_in,
                        reinterpret_cast<const int32_t*>(dc + cp.o_K), reinterpret_cast<const int64_t*>(dc + cp.o_kw),
                        cp.n_K, cp.t.n_kw, reinterpret_cast<const int32_t*>(dc + cp.o_first),
                        reinterpret_cast<const int32_t*>(dc + cp.o_count), cp.n_rings, reinterpret_cast<double*>(cws),
                        reinterpret_cast<double2*>(cws + xsvs_prefix_bytes(cp.T, cp.t)), r.beta_out, st);
    return e;
}

// Intensities of many trajectories in one persistent contraction and, when
// `req` is given, each trajectory's g2 and XSVS contrast after it; with the
// split precisions all of it is one captured graph.
static xs_status batched_impl(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, int32_t n_traj,
                              xs_precision prec, float* const* I_out, const xs_corr_request* req, cudaStream_t st) {
    if (!ctx || !traj || !grid || !I_out || n_traj < 1) return fail(XS_ERR_INVALID_ARG, "bad batched arguments");
    if (prec == XS_PREC_FP32_DIRECT || prec == XS_PREC_FP32_FACTORED) {
        for (int32_t i = 0; i < n_traj; ++i) {
            if (traj[i].pos_on_host) return fail(XS_ERR_INVALID_ARG, "batched trajectories need device positions");
            xs_status s = intensity_impl(ctx, &traj[i], &grid[i], prec, I_out[i], nullptr, st, 0);
            if (s != XS_OK) return s;
            if (!req) continue;
            const xs_corr_request& r = req[i];
            const int64_t T = traj[i].n_frames;
            const int64_t P = (int64_t)grid[i].nx * grid[i].ny * grid[i].nz;
            if (r.n_tau > 0) {
                s = xs_g2(ctx, I_out[i], T, P, r.taus, r.n_tau, r.g2_out, r.mean_out, st);
                if (s != XS_OK) return s;
            }
            if (r.n_K > 0 && r.n_rings > 0) {
                s = xs_xsvs_contrast(ctx, I_out[i], T, &grid[i], &traj[i].box, r.Ks, r.n_K, r.ring_width, r.n_rings,
                                     r.beta_out, r.ring_count_out, st);
                if (s != XS_OK) return s;
            }
        }
        return XS_OK;
    }
    if (prec != XS_PREC_SPLIT_FP16 && prec != XS_PREC_SPLIT_BF16)
        return fail(XS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    // validate and lay out the phase records of every trajectory
    struct Job {
        int64_t N, T, n_pad;
        double hinv[9];
        GridDesc g;
        size_t rec_off;
        int half_axis = -1;  // >= 0: computed on the half grid v, the rest by mirrors
        GridDesc v;
        size_t half_off = 0;
    };
    std::vector<Job> jobs((size_t)n_traj);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = round_up((int64_t)off, 256);
        off = o + bytes;
        return o;
    };
    for (int32_t i = 0; i < n_traj; ++i) {
        const xs_traj& t = traj[i];
        xs_status s = check_grid(&grid[i]);
        if (s != XS_OK) return s;
        if (t.pos_on_host) return fail(XS_ERR_INVALID_ARG, "trajectory %d: batched positions must be on the device", i);
        if (t.n_atoms < 0 || t.n_frames < 0) return fail(XS_ERR_INVALID_ARG, "trajectory %d: negative size", i);
        if (t.n_atoms > 0 && t.n_frames > 0 && (!t.pos || !t.f))
            return fail(XS_ERR_INVALID_ARG, "trajectory %d: NULL positions", i);
        if (t.n_frames > 0 && grid[i].nx * (int64_t)grid[i].ny * grid[i].nz > 0 && !I_out[i])
            return fail(XS_ERR_INVALID_ARG, "trajectory %d: NULL output", i);
        Job& j = jobs[(size_t)i];
        if (!invert3(t.box.h, j.hinv)) return fail(XS_ERR_INVALID_ARG, "trajectory %d: singular cell matrix", i);
        j.N = t.n_atoms;
        j.T = t.n_frames;
        j.n_pad = round_up(j.N > 0 ? j.N : 1, 64);
        j.g = to_desc(&grid[i]);
        if (j.T > 65535 * 8) return fail(XS_ERR_INVALID_ARG, "trajectory %d: too many frames", i);
        j.rec_off = carve((size_t)j.T * j.n_pad * sizeof(AtomRec));
        if (j.N > 0 && j.T > 0 && j.g.pixels() > 0) {
            j.half_axis = friedel_half_grid(j.g, j.v);
            if (j.half_axis >= 0) j.half_off = carve((size_t)j.T * j.v.pixels() * sizeof(float));
        }
    }
    const int cap = std::max(tc_pair_capacity(ctx->num_sms, kTcTile128), tc_pair_capacity(ctx->num_sms, kTcTile64));
    const size_t o_scratch = carve(tc_scratch_bytes(cap));

    // trajectory table and per-pair unit lists (longest first)
    std::vector<TcTraj> trs;
    std::vector<int> which;  // trajectory index of each table entry
    std::vector<int> empty;  // trajectories without atoms: I = 0
    for (int32_t i = 0; i < n_traj; ++i) {
        const Job& j = jobs[(size_t)i];
        if (j.T == 0 || j.g.pixels() == 0) continue;
        if (j.N == 0) {
            empty.push_back(i);
            continue;
        }
        which.push_back(i);
    }
    std::vector<char> blob;
    // correlation requests: host tables into the blob, one shared workspace
    std::vector<CorrPrep> corr(req ? (size_t)n_traj : 0);
    size_t corr_ws = 0;
    for (int32_t i = 0; req && i < n_traj; ++i) {
        xs_status s = corr_prepare(req[i], i, traj[i].n_frames, &grid[i], &traj[i].box, blob, corr[(size_t)i]);
        if (s != XS_OK) return s;
        corr_ws = std::max(corr_ws, corr[(size_t)i].ws_bytes);
    }
    const size_t o_corr = carve(corr_ws);
    xs_status s = ensure_ws(ctx, off + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    // each trajectory's tile kind and chunk length: tuned for its shape
    // bucket (xs_tune), else the default rule; half grids use 128 x 128 tiles
    for (int i : which) {
        const Job& j = jobs[(size_t)i];
        const GridDesc& gc = j.half_axis >= 0 ? j.v : j.g;
        int kind = j.half_axis >= 0 ? kTcTile128 : tc_default_kind(gc), chunk = 0;
        auto it = ctx->tuned.find(tc_bucket(j.n_pad, gc, (int)prec));
        if (it != ctx->tuned.end()) {
            chunk = it->second.chunk;
            if (j.half_axis < 0) kind = it->second.kind;
        }
        if (j.half_axis >= 0)
            trs.push_back(tc_traj(reinterpret_cast<AtomRec*>(ws + j.rec_off), j.n_pad, j.T, j.v,
                                  reinterpret_cast<float*>(ws + j.half_off), nullptr, kind, chunk, ctx->exact_tables));
        else
            trs.push_back(tc_traj(reinterpret_cast<AtomRec*>(ws + j.rec_off), j.n_pad, j.T, j.g, I_out[i], nullptr,
                                  kind, chunk, ctx->exact_tables));
    }
    for (int i : empty)
        XS_CUDA(cudaMemsetAsync(I_out[i], 0, (size_t)jobs[(size_t)i].T * jobs[(size_t)i].g.pixels() * sizeof(float), st));
    if (trs.empty() && !req) return XS_OK;
    // one persistent launch per tile kind, each over the units of its
    // trajectories (entries of the one trajectory table), longest first
    struct KindLaunch {
        int kind, n_pairs = 0;
        size_t o_units = 0, o_ps = 0;
    };
    std::vector<KindLaunch> kls;
    size_t o_tr = 0;
    if (!trs.empty()) {
        o_tr = push(blob, trs.data(), trs.size());
        for (int kind : {kTcTile128, kTcTile64}) {
            std::vector<int4> all;
            for (size_t e = 0; e < trs.size(); ++e) {
                const TcTraj& t = trs[e];
                if (t.kind != kind) continue;
                for (int f = 0; f < t.n_frames; ++f)
                    for (int z = 0; z < t.nz; ++z)
                        for (int ty = 0; ty < t.tiles_y; ++ty)
                            for (int tx = 0; tx < t.tiles_x; ++tx)
                                all.push_back(make_int4((int)e, f, z, tx | (ty << 16)));
            }
            if (all.empty()) continue;
            if (all.size() > (size_t)INT32_MAX) return fail(XS_ERR_UNSUPPORTED, "too many work units");
            KindLaunch kl;
            kl.kind = kind;
            kl.n_pairs = (int)std::min<int64_t>(tc_pair_capacity(ctx->num_sms, kind), (int64_t)all.size());
            std::vector<int4> units;
            std::vector<int> pair_start;
            tc_deal_units(trs, all, kl.n_pairs, units, pair_start);
            kl.o_units = push(blob, units.data(), units.size());
            kl.o_ps = push(blob, pair_start.data(), pair_start.size());
            kls.push_back(kl);
        }
    }
    if (blob.empty()) blob.assign(256, 0);
    void* d = nullptr;
    s = upload_const(ctx, "tc_batch", blob, st, &d);
    if (s != XS_OK) return s;
    char* dc = static_cast<char*>(d);
    const int chunk = kDefaultChunkStages;  // for trajectories without a tuned chunk
    const bool bf16 = prec == XS_PREC_SPLIT_BF16;
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t err = cudaSuccess;
        for (size_t e = 0; e < trs.size() && err == cudaSuccess; ++e) {
            const Job& j = jobs[(size_t)which[e]];
            const xs_traj& t = traj[which[e]];
            Mat3 hm;
            for (int k = 0; k < 9; ++k) hm.a[k] = j.hinv[k];
            PhaseOpts popt;
            popt.ortho = is_ortho(j.hinv);
            const GridDesc& gc = j.half_axis >= 0 ? j.v : j.g;
            popt.need_z = !(gc.nz == 1 && gc.nz0 == 0);
            popt.perm_mul = coprime_stride(j.n_pad / kPermRun);
            err = launch_phase(t.pos, t.f, j.N, j.T, j.n_pad, hm, popt, reinterpret_cast<AtomRec*>(ws + j.rec_off),
                               ctx->d_err, st);
        }
        for (size_t k = 0; k < kls.size() && err == cudaSuccess; ++k)
            err = launch_tc_batch(reinterpret_cast<const TcTraj*>(dc + o_tr),
                                  reinterpret_cast<const int4*>(dc + kls[k].o_units),
                                  reinterpret_cast<const int*>(dc + kls[k].o_ps), kls[k].n_pairs, chunk, bf16,
                                  kls[k].kind, ctx->exact_tables, reinterpret_cast<double*>(ws + o_scratch),
                                  ctx->d_err, ctx->timeout_ns, st);
        for (size_t e = 0; e < trs.size() && err == cudaSuccess; ++e) {
            const Job& j = jobs[(size_t)which[e]];
            if (j.half_axis >= 0)
                err = launch_friedel(reinterpret_cast<const float*>(ws + j.half_off), nullptr, j.T, j.v, j.g,
                                     j.half_axis, I_out[which[e]], nullptr, st);
        }
        // each trajectory's g2 and XSVS contrast, one after another in the
        // shared correlation workspace
        for (int32_t i = 0; req && i < n_traj && err == cudaSuccess; ++i)
            err = corr_launch(corr[(size_t)i], req[i], I_out[i], dc, ws + o_corr, st);
        return err;
    };
    // the same batch (same tables, inputs, outputs and workspace) replays a
    // captured graph; anything else is captured once and kept
    std::string key(blob.begin(), blob.end());
    for (int32_t i = 0; i < n_traj; ++i) {
        const void* ptrs[3] = {traj[i].pos, traj[i].f, I_out[i]};
        key.append(reinterpret_cast<const char*>(ptrs), sizeof(ptrs));
        key.append(reinterpret_cast<const char*>(traj[i].box.h), sizeof(traj[i].box.h));
        if (req) {
            const void* outs[3] = {req[i].g2_out, req[i].mean_out, req[i].beta_out};
            key.append(reinterpret_cast<const char*>(outs), sizeof(outs));
        }
    }
    key.append(reinterpret_cast<const char*>(&chunk), sizeof(chunk));
    key.append(reinterpret_cast<const char*>(&ctx->timeout_ns), sizeof(ctx->timeout_ns));
    key.append(bf16 ? "b" : "h");
    key.append(req ? "c" : "i");
    const void* wsp = ctx->ws;
    key.append(reinterpret_cast<const char*>(&wsp), sizeof(wsp));
    const cudaError_t launched = traced(ctx, "batched", st, [&]() -> cudaError_t {
        auto it = ctx->graphs.find(key);
        if (it == ctx->graphs.end() && st != nullptr) {
            cudaGraph_t graph = nullptr;
            const int64_t before = tl_kernel_launches;
            cudaError_t err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                const cudaError_t le = enqueue();
                err = cudaStreamEndCapture(st, &graph);
                if (le != cudaSuccess) err = le;
            }
            const int64_t captured = tl_kernel_launches - before;
            tl_kernel_launches = before;  // counted again at each replay
            cudaGraphExec_t exec = nullptr;
            if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (err != cudaSuccess) {
                cudaGetLastError();
                return err;
            }
            it = ctx->graphs.emplace(key, xs_context::Graph{exec, captured}).first;
        }
        if (it == ctx->graphs.end()) return enqueue();  // legacy default stream: no capture
        tl_kernel_launches += it->second.kernels;
        return cudaGraphLaunch(it->second.exec, st);
    });
    if (launched != cudaSuccess) return fail(XS_ERR_CUDA, "batched launch: %s", cudaGetErrorString(launched));
    return XS_OK;
}

xs_status xs_intensity_batched(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, int32_t n_traj,
                               xs_precision prec, float* const* I_out, void* cuda_stream) {
    return batched_impl(ctx, traj, grid, n_traj, prec, I_out, nullptr, static_cast<cudaStream_t>(cuda_stream));
}

xs_status xs_xpcs_batched(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, int32_t n_traj,
                          xs_precision prec, float* const* I_out, const xs_corr_request* req, void* cuda_stream) {
    if (!req) return fail(XS_ERR_INVALID_ARG, "req is required");
    return batched_impl(ctx, traj, grid, n_traj, prec, I_out, req, static_cast<cudaStream_t>(cuda_stream));
}

// --------------------------------------------------------------------------
// intermediate scattering function and the contrast it predicts
// --------------------------------------------------------------------------

xs_status xs_isf(xs_context* ctx, const float* amp, int64_t T, int64_t P, const int32_t* taus, int32_t n_tau,
                 double sum_f2, double* F_out, double* Fhat_out, void* cuda_stream) {
    if (!ctx || !amp || !taus || !F_out) return fail(XS_ERR_INVALID_ARG, "context, amp, taus and F_out are required");
    if (T < 1 || P < 0 || n_tau < 0) return fail(XS_ERR_INVALID_ARG, "need T >= 1, P >= 0, n_tau >= 0");
    if (!(sum_f2 > 0.0) || !std::isfinite(sum_f2)) return fail(XS_ERR_INVALID_ARG, "sum_f2 must be finite and > 0");
    for (int32_t k = 0; k < n_tau; ++k)
        if (taus[k] < 0 || taus[k] >= T) return fail(XS_ERR_INVALID_ARG, "delay %d outside [0, T)", taus[k]);
    if (P == 0 || n_tau == 0) return XS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<char> blob;
    const size_t o_tau = push(blob, taus, (size_t)n_tau);
    void* d = nullptr;
    xs_status s = upload_const(ctx, "isf", blob, st, &d);
    if (s != XS_OK) return s;
    const int32_t* d_taus = reinterpret_cast<const int32_t*>(static_cast<char*>(d) + o_tau);
    XS_CUDA(traced(ctx, "isf", st,
                   [&] { return launch_isf(amp, T, P, d_taus, n_tau, 1.0 / sum_f2, F_out, Fhat_out, st); }));
    return XS_OK;
}

xs_status xs_contrast_from_isf(xs_context* ctx, const double* Fhat, int64_t Kmax, const xs_qgrid* grid,
                               const xs_box* box, const int32_t* Ks, int32_t n_K, double ring_width,
                               int32_t n_rings, double* ratio_out, int32_t* ring_count_out, void* cuda_stream) {
    const bool empty = n_K == 0 || n_rings == 0;
    if (!ctx || !Fhat || !box || (!Ks && n_K > 0) || (!ratio_out && !empty))
        return fail(XS_ERR_INVALID_ARG, "missing argument");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (Kmax < 1 || n_K < 0 || n_rings < 0) return fail(XS_ERR_INVALID_ARG, "need Kmax >= 1, n_K >= 0, n_rings >= 0");
    if (!(ring_width > 0.0 && ring_width <= 1.0)) return fail(XS_ERR_INVALID_ARG, "ring_width must be in (0, 1]");
    for (int32_t k = 0; k < n_K; ++k)
        if (Ks[k] < 1 || Ks[k] > Kmax) return fail(XS_ERR_INVALID_ARG, "window length %d outside [1, Kmax]", Ks[k]);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    RingLayout lay;
    s = ring_layout(grid, box, ring_width, n_rings, lay);
    if (s != XS_OK) return s;
    if (ring_count_out && n_rings > 0) std::memcpy(ring_count_out, lay.count.data(), lay.count.size() * sizeof(int32_t));
    if (n_K == 0 || n_rings == 0) return XS_OK;
    const int64_t P = (int64_t)grid->nx * grid->ny * grid->nz;
    const int64_t n_in = lay.start[(size_t)n_rings];
    // window lengths in ascending order, each with its output row
    std::vector<int32_t> order((size_t)n_K);
    for (int32_t k = 0; k < n_K; ++k) order[(size_t)k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return Ks[a] < Ks[b]; });
    std::vector<int32_t> k_sorted((size_t)n_K), k_row((size_t)n_K);
    for (int32_t k = 0; k < n_K; ++k) {
        k_sorted[(size_t)k] = Ks[order[(size_t)k]];
        k_row[(size_t)k] = order[(size_t)k];
    }
    std::vector<char> blob;
    const int64_t key[2] = {Kmax, P};
    push(blob, key, 2);
    const size_t o_perm = push(blob, lay.perm.data(), lay.perm.size());
    const size_t o_start = push(blob, lay.start.data(), lay.start.size());
    const size_t o_K = push(blob, k_sorted.data(), k_sorted.size());
    const size_t o_row = push(blob, k_row.data(), k_row.size());
    void* d = nullptr;
    s = upload_const(ctx, "isf_contrast", blob, st, &d);
    if (s != XS_OK) return s;
    char* dc = static_cast<char*>(d);
    s = ensure_ws(ctx, (size_t)std::max<int64_t>(1, (int64_t)n_K * n_in) * sizeof(double) + 256);
    if (s != XS_OK) return s;
    double* b_pixel = static_cast<double*>(ctx->ws);
    XS_CUDA(traced(ctx, "isf_contrast", st, [&] {
        return launch_isf_contrast(Fhat, Kmax, P, reinterpret_cast<const int32_t*>(dc + o_perm), n_in,
                                   reinterpret_cast<const int32_t*>(dc + o_K), reinterpret_cast<const int32_t*>(dc + o_row),
                                   n_K, reinterpret_cast<const int64_t*>(dc + o_start), n_rings, b_pixel, ratio_out, st);
    }));
    return XS_OK;
}

// --------------------------------------------------------------------------
// adjoint
// --------------------------------------------------------------------------

xs_status xs_intensity_backward(xs_context* ctx, const xs_traj* traj, const xs_qgrid* grid, const float* amp,
                                const float* dL_dI, float* dL_dr_out, void* cuda_stream) {
    if (!ctx || !traj || !amp || !dL_dI || !dL_dr_out) return fail(XS_ERR_INVALID_ARG, "missing argument");
    xs_status s = check_grid(grid);
    if (s != XS_OK) return s;
    if (traj->n_frames != 1) return fail(XS_ERR_INVALID_ARG, "the adjoint takes exactly one frame");
    if (traj->pos_on_host) return fail(XS_ERR_INVALID_ARG, "the adjoint needs device positions");
    if (traj->n_atoms < 0) return fail(XS_ERR_INVALID_ARG, "negative atom count");
    if (traj->n_atoms == 0) return XS_OK;
    if (!traj->pos || !traj->f) return fail(XS_ERR_INVALID_ARG, "positions or form factors are NULL");
    double hinv[9];
    if (!invert3(traj->box.h, hinv)) return fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const GridDesc g = to_desc(grid);
    const int64_t N = traj->n_atoms;
    const int64_t n_pad = round_up(N, 64);
    if (g.pixels() == 0) {
        XS_CUDA(cudaMemsetAsync(dL_dr_out, 0, (size_t)N * 3 * sizeof(float), st));
        return XS_OK;
    }
    Mat3 hm;
    for (int i = 0; i < 9; ++i) hm.a[i] = hinv[i];
    PhaseOpts popt;
    popt.ortho = is_ortho(hinv);
    popt.need_z = !(g.nz == 1 && g.nz0 == 0);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = round_up((int64_t)off, 256);
        off = o + bytes;
        return o;
    };
    const size_t o_rec = carve((size_t)n_pad * sizeof(AtomRec));
    const size_t o_h = carve(adjoint_workspace_bytes(g, n_pad));
    s = ensure_ws(ctx, off + 256);
    if (s != XS_OK) return s;
    char* ws = static_cast<char*>(ctx->ws);
    AtomRec* rec = reinterpret_cast<AtomRec*>(ws + o_rec);
    XS_CUDA(traced(ctx, "phase", st, [&] { return launch_phase(traj->pos, traj->f, N, 1, n_pad, hm, popt, rec, ctx->d_err, st); }));
    XS_CUDA(traced(ctx, "adjoint", st, [&] { return launch_adjoint(rec, N, n_pad, g, hm, amp, dL_dI, ws + o_h, dL_dr_out, ctx->d_err,
                                                                           ctx->timeout_ns, st); }));
    return XS_OK;
}

}  // extern "C"
