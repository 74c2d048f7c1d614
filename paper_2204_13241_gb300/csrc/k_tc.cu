// Tensor-core form of the direct method (Algorithm 1, Sec. 3.1).
//
// For q on the reciprocal lattice (q = 2 pi h^-T n, Sec. 3.1) the phase of
// atom j factorises over the axes:
//   exp(i q.r_j) = E_x[n_x](j) E_y[n_y](j) E_z[n_z](j),  E_a[n](j) = exp(i 2 pi n s_ja),
// so the amplitude of one detector plane is a complex contraction over atoms
//   S(n_x, n_y) = sum_j E_x[n_x](j) * w_j(n_y),   w_j(n_y) = f_j E_z[n_z](j) E_y[n_y](j).
// Rows of A are Re and Im of E_x[n_x], rows of B are Re and Im of w(n_y); within
// each group of 4 rows the order is (Re n, Re n+1, Im n, Im n+1) for even n.
// The real product D = A B^T holds the four real partial sums:
//   Re S = D[Re x][Re y] - D[Im x][Im y],  Im S = D[Re x][Im y] + D[Im x][Re y].
//
// One CTA owns a tile of 64 n_x by 128 n_y of one frame and plane
// (MMA M = 128, N = 256) and loops over all atoms 32 at a time (a stage):
//   * 6 producer warps write the factor tables straight into shared memory in
//     the MN-major, 128-byte-swizzled layout the tensor core reads.  Each
//     thread owns one atom and a run of 32 consecutive n, held as pairs
//     (n, n+1) in packed FP32x2 registers (real parts together, imaginary
//     parts together): the run starts from exact seeds exp(i 2 pi n0 U) and
//     exp(i 2 pi (n0+1) U) (U = 32-bit turn count, n U mod 2^32 is exact) and
//     advances by the exact step exp(i 2 pi 2U).  Each value c is split into
//     hi = RN(c) and lo = RN(c - hi) (FP16 or BF16).
//   * 1 thread issues tcgen05.mma (hi*hi + hi*lo + lo*hi, FP32 accumulate)
//     into one of two TMEM accumulators; after `chunk_stages` stages it hands
//     the accumulator to the epilogue and continues in the other one.
//   * 4 epilogue warps add each chunk's FP32 sums into FP64 running totals in
//     an L2-resident scratch buffer (one per CTA) and, after the last chunk of
//     a tile, recombine the quadrants in FP64 into S and I = |S|^2.
// The atoms arrive in a coprime-stride permuted order (see the phase kernel),
// so the partial sums over a chunk behave like random walks even for ordered
// crystals and the FP32 accumulator never sums a coherent run of terms.
// Every wait is bounded: on expiry the kernel sets the device error word and
// all roles leave their loops; tensor memory is released in every case.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kBM = 128;   // MMA M: 64 complex n_x as interleaved Re/Im rows
constexpr int kBN = 256;   // MMA N: 128 complex n_y as interleaved Re/Im columns
constexpr int kBK = 32;    // atoms per stage
constexpr int kStages = 4;
constexpr int kTileX = 64;
constexpr int kTileY = 128;
constexpr int kRun = 32;   // consecutive n per producer thread and stage
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kProdWarps = 6;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;
// MN-major SW128 tiles: blocks of 64 MN elements (128-byte rows), 8 K rows per
// 1024-byte swizzle atom; a stage holds kBK / 8 = 4 K atoms per MN block.
constexpr uint32_t kKAtoms = kBK / 8;
constexpr uint32_t kMNBlockBytes = kKAtoms * 1024;                // 4 KB: LBO
constexpr uint32_t kABytes = (kBM / 64) * kMNBlockBytes;          // 8 KB
constexpr uint32_t kBBytes = (kBN / 64) * kMNBlockBytes;          // 16 KB
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;       // 48 KB
constexpr uint32_t kTmemCols = 512;  // two 256-column FP32 accumulators

struct SmemCtl {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

constexpr size_t kSmemBytes = 1024 + kStages * kStageBytes + sizeof(SmemCtl);

struct TcArgs {
    const uint4* rec;
    int64_t n_pad;
    int n_frames;
    GridDesc g;
    int tiles_x, tiles_y;
    int64_t n_units;
    int n_stages;
    int chunk_stages;
    float* I;
    float* amp;
    double* scratch;  // [gridDim.x][256][128] FP64 running totals
    int* err;
    int64_t timeout_ns;
};

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

// Test of the phase with parity `parity`; the thread may sleep in the barrier
// for up to `hint_ns` before the answer comes back (no busy issue slots).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T; accumulate unless acc == 0
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                     uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on `bar` once every tcgen05 operation issued so far by this thread completes
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 columns of this warp's 32 TMEM lanes; the registers are valid only after
// tmem_wait16 on them (which carries the data dependency for the compiler)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Shared-memory matrix descriptor, MN-major with 128-byte swizzle: leading
// byte offset = stride between 64-element MN blocks, stride byte offset =
// stride between 8-row K atoms (1024 B).
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kMNBlockBytes >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 D, A and B FP16 (or BF16), both MN-major.
__host__ __device__ constexpr uint32_t make_idesc(bool bf16, int M, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bounded wait; false if aborted or timed out (which also raises the abort flag)
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int64_t timeout_ns,
                         uint32_t hint_ns) {
    if (mbar_try_wait(bar, parity, 0u)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity, hint_ns)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(globaltimer_ns() - t0) > timeout_ns) {
            *abort_flag = 1;
            set_dev_error(err, kDevErrTimeout);
            return false;
        }
    }
}

// ---- table construction ------------------------------------------------------

// v = (v0, v1) -> packed hi = (RN(v0), RN(v1)) and lo = (RN(v0 - hi0), RN(v1 - hi1));
// v - hi is exact in FP32, so hi + lo carries about twice the format's bits
template <bool BF16>
__device__ __forceinline__ void split2(float2 v, uint32_t& hi, uint32_t& lo) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        const float2 d = __ffma2_rn(__bfloat1622float2(h), make_float2(-1.0f, -1.0f), v);
        const __nv_bfloat162 l = __float22bfloat162_rn(d);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __float22half2_rn(v);
        const float2 d = __ffma2_rn(__half22float2(h), make_float2(-1.0f, -1.0f), v);
        const __half2 l = __float22half2_rn(d);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// byte offset of the 16-byte chunk holding MN rows [mn, mn+8) of K row k
__device__ __forceinline__ uint32_t chunk_off(int mn, int k) {
    return (uint32_t)(mn >> 6) * kMNBlockBytes + (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * 128u +
           ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4);
}

struct UnitPos {
    int t, iz, tx, ty;
};

__device__ __forceinline__ UnitPos decode_unit(int64_t u, const TcArgs& a) {
    UnitPos p;
    p.tx = (int)(u % a.tiles_x);
    int64_t r = u / a.tiles_x;
    p.ty = (int)(r % a.tiles_y);
    r /= a.tiles_y;
    p.iz = (int)(r % a.g.nz);
    p.t = (int)(r / a.g.nz);
    return p;
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) tc_kernel(TcArgs args) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* smem = smem_raw + pad;
    const uint32_t stage_base = smem_u32(smem);
    SmemCtl* ctl = reinterpret_cast<SmemCtl*>(smem + kStages * kStageBytes);
    volatile int* abort_flag = &ctl->abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == kMmaWarp * 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&ctl->full[s], kProdThreads);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->acc_full[b], 1);
            mbar_init(&ctl->acc_empty[b], kEpiWarps * 32);
        }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&ctl->tmem_base, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    const int64_t my_units =
        args.n_units > blockIdx.x ? (args.n_units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int n_chunks = (args.n_stages + args.chunk_stages - 1) / args.chunk_stages;

    if (warp >= kMmaWarp + 1) {
        // ------------------------------------------------------------ producers
        // warp seg 0,1: A rows for n_x run [32 seg, +32); seg 2..5: B rows for
        // n_y run [32 (seg-2), +32); lane = atom of the stage
        const int seg = warp - (kMmaWarp + 1);
        const bool is_a = seg < 2;
        const int run0 = (is_a ? seg : seg - 2) * kRun;
        const int k = lane;
        const int n_st = args.n_stages;
        int slot = 0;
        uint32_t phase = 0;  // parity of the current pass over the ring of stages
        // records are prefetched one stage ahead; positions of the next tile
        // are decoded once per tile (no integer division inside the stage loop)
        const uint4* rec_cur = nullptr;
        UnitPos up{};
        if (my_units > 0) {
            up = decode_unit(blockIdx.x, args);
            rec_cur = args.rec + (int64_t)up.t * args.n_pad + k;
        }
        uint4 r_next = make_uint4(0, 0, 0, 0);
        if (my_units > 0) r_next = __ldg(rec_cur);
        bool stop = false;
        for (int64_t ku = 0; ku < my_units && !stop; ++ku) {
            UnitPos up_next{};
            const uint4* rec_next_unit = nullptr;
            if (ku + 1 < my_units) {
                up_next = decode_unit(blockIdx.x + (ku + 1) * gridDim.x, args);
                rec_next_unit = args.rec + (int64_t)up_next.t * args.n_pad + k;
            }
            const uint32_t n0 = is_a ? (uint32_t)(args.g.nx0 + up.tx * kTileX + run0)
                                     : (uint32_t)(args.g.ny0 + up.ty * kTileY + run0);
            const uint32_t nz = (uint32_t)(args.g.nz0 + up.iz);
            for (int s = 0; s < n_st; ++s) {
                const uint4 r = r_next;
                if (s + 1 < n_st)
                    r_next = __ldg(rec_cur + (int64_t)(s + 1) * kBK);
                else if (rec_next_unit)
                    r_next = __ldg(rec_next_unit);
                // exact step z^2 and seeds E(n0), E(n0 + 1) of this thread's run
                const uint32_t U = is_a ? r.x : r.y;
                float c, sn;
                phase_to_cs(2u * U, c, sn);
                const float2 ZR = make_float2(c, c), ZI = make_float2(sn, sn), NZI = make_float2(-sn, -sn);
                phase_to_cs(n0 * U, c, sn);
                float2 E0 = make_float2(c, sn);
                phase_to_cs((n0 + 1u) * U, c, sn);
                float2 E1 = make_float2(c, sn);
                if (!is_a) {
                    const float f = __uint_as_float(r.w);
                    float2 w = make_float2(f, 0.0f);
                    if (nz != 0u) {
                        phase_to_cs(nz * r.z, c, sn);
                        w = make_float2(f * c, f * sn);
                    }
                    E0 = cmul(E0, w);
                    E1 = cmul(E1, w);
                }
                float2 R = make_float2(E0.x, E1.x);   // Re of (n, n+1)
                float2 Im = make_float2(E0.y, E1.y);  // Im of (n, n+1)
                if (!wait_bar(&ctl->empty[slot], phase ^ 1u, abort_flag, args.err, args.timeout_ns, 20000u)) {
                    stop = true;
                    break;
                }
                const uint32_t sb = stage_base + (uint32_t)slot * kStageBytes;
                const uint32_t hi_base = is_a ? sb : sb + 2 * kABytes;
                const uint32_t lo_base = hi_base + (is_a ? kABytes : kBBytes);
#pragma unroll
                for (int g = 0; g < kRun / 4; ++g) {
                    // one 16-byte chunk = rows (Re n, Re n+1, Im n, Im n+1, Re n+2, Re n+3, Im n+2, Im n+3)
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        split2<BF16>(R, h[2 * q], l[2 * q]);
                        split2<BF16>(Im, h[2 * q + 1], l[2 * q + 1]);
                        const float2 Rn = __ffma2_rn(R, ZR, __fmul2_rn(Im, NZI));
                        Im = __ffma2_rn(R, ZI, __fmul2_rn(Im, ZR));
                        R = Rn;
                    }
                    const uint32_t off = chunk_off(2 * (run0 + 4 * g), k);
                    st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
                    st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
                }
                fence_async_shared();
                mbar_arrive(&ctl->full[slot]);
                if (++slot == kStages) {
                    slot = 0;
                    phase ^= 1u;
                }
            }
            up = up_next;
            rec_cur = rec_next_unit;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = make_idesc(BF16, kBM, kBN);
            int64_t a_cnt = 0;
            int slot = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t ku = 0; ku < my_units && ok; ++ku) {
                for (int c = 0; c < n_chunks && ok; ++c, ++a_cnt) {
                    const int b = (int)(a_cnt & 1);
                    const uint32_t use = (uint32_t)(a_cnt >> 1);
                    if (!wait_bar(&ctl->acc_empty[b], (use & 1u) ^ 1u, abort_flag, args.err, args.timeout_ns,
                                  20000u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)b * 256u;
                    const int s0 = c * args.chunk_stages;
                    const int s1 = min(args.n_stages, s0 + args.chunk_stages);
                    for (int s = s0; s < s1; ++s) {
                        if (!wait_bar(&ctl->full[slot], phase, abort_flag, args.err, args.timeout_ns, 20000u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_hi = stage_base + (uint32_t)slot * kStageBytes;
                        const uint32_t a_lo = a_hi + kABytes;
                        const uint32_t b_hi = a_hi + 2 * kABytes;
                        const uint32_t b_lo = b_hi + kBBytes;
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint32_t ko = (uint32_t)kk * 2048u;  // two 8-row K atoms per K = 16
                            umma(d_tmem, mn_desc(a_hi + ko), mn_desc(b_hi + ko), idesc, (s > s0 || kk > 0) ? 1u : 0u);
                            umma(d_tmem, mn_desc(a_hi + ko), mn_desc(b_lo + ko), idesc, 1u);
                            umma(d_tmem, mn_desc(a_lo + ko), mn_desc(b_hi + ko), idesc, 1u);
                        }
                        umma_commit(&ctl->empty[slot]);
                        if (++slot == kStages) {
                            slot = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) umma_commit(&ctl->acc_full[b]);
                }
            }
            // every issued MMA must finish before tensor memory is released
            umma_commit(&ctl->drain);
            int no_abort = 0;
            wait_bar(&ctl->drain, 0u, &no_abort, args.err, 2000000000LL, 20000u);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        // TMEM lane = A row; rows 4g..4g+3 are (Re x, Re x+1, Im x, Im x+1), x = 2g
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const int row = warp * 32 + lane;
        const bool re_row = (lane & 2) == 0;
        const int xi = 2 * (row >> 2) + (row & 1);
        double* scr = args.scratch + (size_t)blockIdx.x * 256 * 128 + row;
        int64_t a_cnt = 0;
        bool ok = true;
        for (int64_t ku = 0; ku < my_units && ok; ++ku) {
            const UnitPos up = decode_unit(blockIdx.x + ku * gridDim.x, args);
            for (int c = 0; c < n_chunks; ++c, ++a_cnt) {
                const int b = (int)(a_cnt & 1);
                const uint32_t use = (uint32_t)(a_cnt >> 1);
                uint32_t got = 0;
                if (lane == 0)
                    got = wait_bar(&ctl->acc_full[b], use & 1u, abort_flag, args.err, args.timeout_ns, 200000u);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = lane_base + (uint32_t)b * 256u;
                const bool first = c == 0, last = c == n_chunks - 1;
#pragma unroll 1
                for (int j = 0; j < kBN / 16; ++j) {
                    uint32_t r[16];
                    tmem_ld16(dcol + 16 * j, r);
                    tmem_wait16(r);
                    double v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        v[i] = (double)__uint_as_float(r[i]);
                        if (!first) v[i] += scr[(size_t)(16 * j + i) * 128];
                    }
                    if (!last) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) scr[(size_t)(16 * j + i) * 128] = v[i];
                        continue;
                    }
                    // columns 16j .. 16j+15 hold n_y local m = 8j .. 8j+7 in groups of 4
                    // (Re m, Re m+1, Im m, Im m+1); the Re lane finishes m = 8j..8j+3 with
                    // the Im values of its partner lane (lane ^ 2), the Im lane m = 8j+4..8j+7
                    double own[8], rcv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        own[i] = re_row ? v[i] : v[8 + i];
                        const double snd = re_row ? v[8 + i] : v[i];
                        rcv[i] = __shfl_xor_sync(0xffffffffu, snd, 2);
                    }
                    const int ix = up.tx * kTileX + xi;
                    if (ix < args.g.nx) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const double* vr = re_row ? own : rcv;  // D[Re x][...]
                                const double* vi = re_row ? rcv : own;  // D[Im x][...]
                                const double p_rr = vr[4 * hh + t], p_ri = vr[4 * hh + 2 + t];
                                const double p_ir = vi[4 * hh + t], p_ii = vi[4 * hh + 2 + t];
                                const double sre = p_rr - p_ii;
                                const double sim = p_ri + p_ir;
                                const int m = 8 * j + (re_row ? 0 : 4) + 2 * hh + t;
                                const int iy = up.ty * kTileY + m;
                                if (iy < args.g.ny) {
                                    const int64_t o =
                                        (((int64_t)up.t * args.g.nz + up.iz) * args.g.ny + iy) * args.g.nx + ix;
                                    args.I[o] = (float)(sre * sre + sim * sim);
                                    if (args.amp) {
                                        args.amp[2 * o] = (float)sre;
                                        args.amp[2 * o + 1] = (float)sim;
                                    }
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&ctl->acc_empty[b]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

bool tc_supported(const GridDesc& g) { return g.nx >= 1 && g.ny >= 1 && g.nz >= 1; }

int64_t tc_atom_multiple() { return kBK; }

TcPlan plan_tc(int64_t n_pad, int64_t n_frames, const GridDesc& g, int num_sms, int chunk_stages) {
    TcPlan p;
    p.tiles_x = (g.nx + kTileX - 1) / kTileX;
    p.tiles_y = (g.ny + kTileY - 1) / kTileY;
    const int64_t units = n_frames * g.nz * p.tiles_x * p.tiles_y;
    p.grid = (int)std::min<int64_t>(units, num_sms);
    p.chunk_stages = chunk_stages > 0 ? chunk_stages : 128;
    (void)n_pad;
    return p;
}

size_t tc_scratch_bytes(const TcPlan& plan) { return (size_t)plan.grid * 256 * 128 * sizeof(double); }

cudaError_t launch_tc(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g, const TcPlan& plan,
                      bool bf16, float* I, float* amp, double* scratch, int* err, int64_t timeout_ns,
                      cudaStream_t st) {
    if (n_pad % kBK != 0) return cudaErrorInvalidValue;
    TcArgs a;
    a.rec = reinterpret_cast<const uint4*>(rec);
    a.n_pad = n_pad;
    a.n_frames = (int)n_frames;
    a.g = g;
    a.tiles_x = plan.tiles_x;
    a.tiles_y = plan.tiles_y;
    a.n_units = n_frames * g.nz * plan.tiles_x * plan.tiles_y;
    a.n_stages = (int)(n_pad / kBK);
    a.chunk_stages = plan.chunk_stages;
    a.I = I;
    a.amp = amp;
    a.scratch = scratch;
    a.err = err;
    a.timeout_ns = timeout_ns;
    if (a.n_units == 0) return cudaSuccess;
    const void* fn = bf16 ? (const void*)tc_kernel<true> : (const void*)tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    ++tl_kernel_launches;
    if (bf16)
        tc_kernel<true><<<plan.grid, kThreads, kSmemBytes, st>>>(a);
    else
        tc_kernel<false><<<plan.grid, kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace xs
