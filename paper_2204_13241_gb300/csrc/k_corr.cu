// Correlation stages on the intensity series I[t][p]:
//   g2 (Sec. 2.3, Eq. g2_def) and the XSVS contrast (Eqs. inte_Iq, bq_Iq).
//
// g2_series_kernel (series of up to 3,200 frames): a block copies the whole
//   series of W consecutive pixels into shared memory once (W = 32 up to
//   1,600 frames, 16 up to 3,200, so that they fit in 200 KB),
//   then each thread sums one pixel's products for a group of up to 4 delays
//   (2 on 16 pixels) and the first group also the pixel's mean, all read from
//   shared memory.
//   Products are summed in plain FP32 over 8 frames (a relative error of at
//   most 7 eps for these positive terms), those sums with compensated FP32
//   over 256-frame blocks, the block sums in FP64.  Each operand is read from
//   HBM once instead of once per delay from L2, and a product costs a load
//   and an FMA instead of a load and four compensated operations.
//
// g2_kernel (longer series): one thread per pixel, group of up to kTauGroup delays and
//   segment of frames (blockIdx.z).  The block walks its frames t in order;
//   I[t][p] and I[t+tau][p] are coalesced across the pixels of a warp.
//   Products and the mean (summed by the blocks of the first delay group)
//   are summed with compensated (Kahan) FP32 updates over blocks of up to 256
//   frames, and the block sums are added in FP64.  Frames whose delays all
//   stay inside the series run a loop with one pointer step per frame and a
//   precomputed offset per delay, without bound checks.  Each segment writes FP64
//   partial sums; g2_finish_kernel adds the segments in order and divides.
//   The segments (up to 8, each a whole number of 64-frame blocks) give the
//   kernel more blocks.
//
// XSVS: pixels are first permuted ring by ring (host-built permutation), then
//   segment_total_kernel, prefix_kernel
//                   C[t][p'] = sum_{t'<t} I[t'][perm[p']]       (FP64, [T+1][P'])
//                   over up to 8 frame segments in parallel
//   window_kernel   per (ring chunk, (K,w)): sum_p x and sum_p x^2 with
//                   x = C[(w+1)K][p'] - C[wK][p'] (one warp per 8 (K,w))
//   finalize_kernel per (K, ring): ring sums over the ring's chunks in a fixed
//                   order, beta per window, mean over windows.
//
// Intermediate scattering function on the amplitude series S[t][p] (Sec. 2.3,
// Eqs. Fq_pq, norm_Fq) and the contrast it predicts (Eq. beta_alt_int):
//   isf_kernel      like g2_kernel with complex products conj(S(t)) S(t+tau)
//                   (compensated FP32 over 256-frame blocks, FP64 block sums),
//                   F = mean / sum f^2 and F_hat = F / F(q,0)
//   isf_contrast_kernel per in-ring pixel, one pass over the delays d:
//                   (1/K^2) [K + 2 (K sum_{d<K} |F_hat|^2 - sum_{d<K} d |F_hat|^2)]
//   ring_mean_kernel per (K, ring), fixed-order mean over the ring's pixels.
#include <algorithm>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kTauGroup = 16;
constexpr int kG2Threads = 128;
constexpr int kFlush = 64;
constexpr int64_t kPrefixSegs = 8;  // frame segments of the XSVS prefix sums
// frames per compensated FP32 block of g2_kernel and isf_kernel before their
// FP64 totals: the FP64 pipe is narrow on GB300, and a compensated sum of up
// to 256 terms stays within about 2 eps of the sum of their magnitudes
constexpr int kG2Flush = 256;

__global__ void __launch_bounds__(kG2Threads)
g2_kernel(const float* __restrict__ I, int64_t T, int64_t P, const int32_t* __restrict__ taus,
          int n_tau, int64_t seg_len, double* __restrict__ part, double* __restrict__ mpart) {
    __shared__ int s_tau[kTauGroup];
    const int g0 = blockIdx.y * kTauGroup;
    const int nt = min(kTauGroup, n_tau - g0);
    if (threadIdx.x < kTauGroup) s_tau[threadIdx.x] = threadIdx.x < nt ? taus[g0 + threadIdx.x] : 0;
    __syncthreads();
    const int64_t p = blockIdx.x * (int64_t)kG2Threads + threadIdx.x;
    if (p >= P) return;
    // offset of I[t + tau_k][p] from I[t][p]; unused delays of a partial
    // group point at I[t][p] itself and are never written out
    int64_t off[kTauGroup];
    int tau_max = 0;
#pragma unroll
    for (int k = 0; k < kTauGroup; ++k) {
        off[k] = (int64_t)s_tau[k] * P;
        tau_max = max(tau_max, s_tau[k]);
    }
    float acc[kTauGroup], comp[kTauGroup];
    double dacc[kTauGroup];
#pragma unroll
    for (int k = 0; k < kTauGroup; ++k) {
        acc[k] = comp[k] = 0.0f;
        dacc[k] = 0.0;
    }
    double dmean = 0.0;
    float macc = 0.0f, mcomp = 0.0f;
    const bool want_mean = blockIdx.y == 0;  // the first delay group sums the mean
    const int64_t seg0 = (int64_t)blockIdx.z * seg_len, seg1 = min(T, seg0 + seg_len);
    for (int64_t t0 = seg0; t0 < seg1; t0 += kG2Flush) {
        const int64_t t1 = min(seg1, t0 + kG2Flush);
        // frames t < T - tau_max have every delay inside the series: the loop
        // over them carries no bound checks and no index arithmetic but one
        // pointer step (the kernel is bound by instruction issue)
        const int64_t tf = max(t0, min(t1, T - (int64_t)tau_max));
        const float* row = I + t0 * P + p;
        int64_t t = t0;
        for (; t < tf; ++t, row += P) {
            const float x = row[0];
            if (want_mean) {
                const float ym = x - mcomp;
                const float sm = macc + ym;
                mcomp = (sm - macc) - ym;
                macc = sm;
            }
#pragma unroll
            for (int k = 0; k < kTauGroup; ++k) {
                const float y = fmaf(x, row[off[k]], -comp[k]);
                const float s = acc[k] + y;
                comp[k] = (s - acc[k]) - y;
                acc[k] = s;
            }
        }
        for (; t < t1; ++t, row += P) {
            const float x = row[0];
            if (want_mean) {
                const float ym = x - mcomp;
                const float sm = macc + ym;
                mcomp = (sm - macc) - ym;
                macc = sm;
            }
#pragma unroll
            for (int k = 0; k < kTauGroup; ++k) {
                if (k < nt && t + s_tau[k] < T) {
                    const float y = fmaf(x, row[off[k]], -comp[k]);
                    const float s = acc[k] + y;
                    comp[k] = (s - acc[k]) - y;
                    acc[k] = s;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kTauGroup; ++k) {
            dacc[k] += (double)acc[k] - (double)comp[k];
            acc[k] = comp[k] = 0.0f;
        }
        dmean += (double)macc - (double)mcomp;
        macc = mcomp = 0.0f;
    }
    const int64_t seg = blockIdx.z;
    if (want_mean) mpart[seg * P + p] = dmean;
#pragma unroll
    for (int k = 0; k < kTauGroup; ++k) {
        if (k < nt) part[(seg * n_tau + g0 + k) * P + p] = dacc[k];
    }
}

constexpr int kG2sMaxPix = 32;     // pixels per block at most: one 128-byte row per frame
constexpr int kG2sThreads = 512;
constexpr int64_t kG2sMaxBytes = 200 * 1024;  // shared memory for the series of a block's pixels
constexpr int kG2sSub = 8;         // frames per plain FP32 sum before the compensated update

// pixels per block for a series of T frames: 32, or 16 where 32 pixels'
// series do not fit in kG2sMaxBytes; 0 (the segment kernel) beyond.  Rows of
// 16 pixels are two full 32-byte sectors; narrower rows made the loads a
// gather of one partial sector per frame and row, and the 10,000-frame
// 512^2 series took 183 ms instead of 150 ms with 4 pixels per block.
int g2s_width(int64_t T) {
    for (int w = kG2sMaxPix; w >= 16; w >>= 1)
        if ((int64_t)w * T * (int64_t)sizeof(float) <= kG2sMaxBytes) return w;
    return 0;
}

// Kahan update: (acc, comp) += v
__device__ __forceinline__ void kahan_add(float& acc, float& comp, float v) {
    const float y = v - comp;
    const float s = acc + y;
    comp = (s - acc) - y;
    acc = s;
}

// frames [t, t + n) of one pixel's series (column `col` of s_x, rows of W
// floats) for up to D delays: the n products per delay are summed in plain
// FP32 (at most 8 terms), then added to the compensated totals.  CHECK:
// frames whose partner t + tau lies past the series, and unused delay slots,
// are skipped.
template <int D, bool CHECK>
__device__ __forceinline__ void g2s_sub(const float* col, int W, int t, int n, int T, const int* tau, const int* off,
                                        int nk, float* acc, float* comp, bool want_mean, float& macc, float& mcomp) {
    float sk[D], sm = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) sk[k] = 0.0f;
#pragma unroll
    for (int u = 0; u < kG2sSub; ++u) {
        if (CHECK && u >= n) break;
        const float* r = col + (t + u) * W;
        const float x = r[0];
        sm += x;
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (!CHECK || (k < nk && t + u + tau[k] < T)) sk[k] = fmaf(x, r[off[k]], sk[k]);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) kahan_add(acc[k], comp[k], sk[k]);
    if (want_mean) kahan_add(macc, mcomp, sm);
}

// W pixels per block (g2s_width), D delays per thread
template <int D>
__global__ void __launch_bounds__(kG2sThreads, 1)
g2_series_kernel(const float* __restrict__ I, int64_t T, int64_t P, const int32_t* __restrict__ taus, int n_tau,
                 int W, double* __restrict__ g2, double* __restrict__ mean_out) {
    extern __shared__ float s_x[];  // [T][W]
    __shared__ double s_mean[kG2sMaxPix];
    const int64_t p0 = (int64_t)blockIdx.x * W;
    const int np = (int)min((int64_t)W, P - p0);
    // asynchronous 4-byte copies, all in flight at once (a loop of loads and
    // stores would wait for each load); pixels past P are filled with zeros
    for (int64_t e = threadIdx.x; e < T * W; e += blockDim.x) {
        const int64_t t = e / W;
        const int i = (int)(e - t * W);
        const float* src = I + t * P + p0 + (i < np ? i : 0);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_x + e);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(i < np ? 4 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int n_groups = (n_tau + D - 1) / D;
    const int Ti = (int)T;
    for (int item = threadIdx.x; item < W * n_groups; item += blockDim.x) {
        const int i = item % W, grp = item / W;
        const int k0 = grp * D, nk = min(D, n_tau - k0);
        int tau[D], off[D];  // off: offset of x(t + tau_k) from x(t) in s_x
        int tau_max = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            tau[k] = k < nk ? taus[k0 + k] : 0;
            off[k] = tau[k] * W;
            tau_max = max(tau_max, tau[k]);
        }
        float acc[D], comp[D];
        double dacc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            acc[k] = comp[k] = 0.0f;
            dacc[k] = 0.0;
        }
        double dmean = 0.0;
        float macc = 0.0f, mcomp = 0.0f;
        const bool want_mean = grp == 0;
        const float* col = s_x + i;
        for (int t0 = 0; t0 < Ti; t0 += kG2Flush) {
            const int t1 = min(Ti, t0 + kG2Flush);
            const int tf = max(t0, min(t1, Ti - tau_max));
            int t = t0;
            for (; t + kG2sSub <= tf; t += kG2sSub)
                g2s_sub<D, false>(col, W, t, kG2sSub, Ti, tau, off, nk, acc, comp, want_mean, macc, mcomp);
            for (; t < t1; t += kG2sSub)
                g2s_sub<D, true>(col, W, t, min(kG2sSub, t1 - t), Ti, tau, off, nk, acc, comp, want_mean, macc,
                                 mcomp);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                dacc[k] += (double)acc[k] - (double)comp[k];
                acc[k] = comp[k] = 0.0f;
            }
            dmean += (double)macc - (double)mcomp;
            macc = mcomp = 0.0f;
        }
        const int64_t p = p0 + i;
        if (want_mean) {
            const double m = dmean / (double)T;
            s_mean[i] = m;
            if (mean_out && i < np) mean_out[p] = m;
        }
        // the numerator's average for now; divided by the squared mean below
        if (i < np) {
#pragma unroll
            for (int k = 0; k < D; ++k)
                if (k < nk) g2[(int64_t)(k0 + k) * P + p] = dacc[k] / (double)(T - taus[k0 + k]);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n_tau * W; e += blockDim.x) {
        const int k = e / W, i = e % W;
        if (i >= np) continue;
        const double m = s_mean[i];
        double* gp = g2 + (int64_t)k * P + p0 + i;
        *gp = *gp / (m * m);
    }
}

template <int D>
cudaError_t launch_g2_series(const float* I, int64_t T, int64_t P, const int32_t* d_taus, int n_tau, int W,
                             double* g2, double* mean, cudaStream_t st) {
    const size_t smem = (size_t)T * W * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(g2_series_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int items = W * ((n_tau + D - 1) / D);
    const int threads = std::min(kG2sThreads, (items + 31) / 32 * 32);
    ++tl_kernel_launches;
    g2_series_kernel<D><<<(unsigned)((P + W - 1) / W), threads, smem, st>>>(I, T, P, d_taus, n_tau, W, g2, mean);
    return cudaGetLastError();
}

// one thread per (delay, pixel): segments added in order
__global__ void g2_finish_kernel(const double* __restrict__ part, const double* __restrict__ mpart, int n_seg,
                                 int64_t T, int64_t P, const int32_t* __restrict__ taus, int n_tau,
                                 double* __restrict__ g2, double* __restrict__ mean_out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_tau * P) return;
    const int k = (int)(i / P);
    const int64_t p = i - (int64_t)k * P;
    double msum = 0.0, sum = 0.0;
    for (int s = 0; s < n_seg; ++s) {
        msum += mpart[(int64_t)s * P + p];
        sum += part[((int64_t)s * n_tau + k) * P + p];
    }
    const double m = msum / (double)T;
    if (k == 0 && mean_out) mean_out[p] = m;
    g2[i] = (sum / (double)(T - taus[k])) / (m * m);
}

constexpr int kIsfGroup = 8;

__global__ void __launch_bounds__(kG2Threads)
isf_kernel(const float2* __restrict__ S, int64_t T, int64_t P, const int32_t* __restrict__ taus, int n_tau,
           double inv_sum_f2, double2* __restrict__ F, double2* __restrict__ Fhat) {
    __shared__ int s_tau[kIsfGroup];
    const int g0 = blockIdx.y * kIsfGroup;
    const int nt = min(kIsfGroup, n_tau - g0);
    if (threadIdx.x < kIsfGroup) s_tau[threadIdx.x] = threadIdx.x < nt ? taus[g0 + threadIdx.x] : 0;
    __syncthreads();
    const int64_t p = blockIdx.x * (int64_t)kG2Threads + threadIdx.x;
    if (p >= P) return;
    // offset of S[t + tau_k][p] from S[t][p]; unused delays of a partial group
    // point at S[t][p] itself and are never written out
    int64_t off[kIsfGroup];
    int tau_max = 0;
#pragma unroll
    for (int k = 0; k < kIsfGroup; ++k) {
        off[k] = (int64_t)s_tau[k] * P;
        tau_max = max(tau_max, s_tau[k]);
    }
    float are[kIsfGroup], cre[kIsfGroup], aim[kIsfGroup], cim[kIsfGroup];
    double dre[kIsfGroup], dim[kIsfGroup];
#pragma unroll
    for (int k = 0; k < kIsfGroup; ++k) {
        are[k] = cre[k] = aim[k] = cim[k] = 0.0f;
        dre[k] = dim[k] = 0.0;
    }
    double dmean = 0.0;
    float macc = 0.0f, mcomp = 0.0f;  // |S|^2, compensated like the products
    auto add_mean = [&](float2 a) {
        const float y = fmaf(a.x, a.x, fmaf(a.y, a.y, -mcomp));
        const float s = macc + y;
        mcomp = (s - macc) - y;
        macc = s;
    };
    // conj(a) b = (a.x b.x + a.y b.y) + i (a.x b.y - a.y b.x), compensated
    auto add = [&](int k, float2 a, float2 b) {
        const float yr = fmaf(a.x, b.x, fmaf(a.y, b.y, -cre[k]));
        const float sr = are[k] + yr;
        cre[k] = (sr - are[k]) - yr;
        are[k] = sr;
        const float yi = fmaf(a.x, b.y, fmaf(-a.y, b.x, -cim[k]));
        const float si = aim[k] + yi;
        cim[k] = (si - aim[k]) - yi;
        aim[k] = si;
    };
    for (int64_t t0 = 0; t0 < T; t0 += kG2Flush) {
        const int64_t t1 = min(T, t0 + kG2Flush);
        // frames whose delays all stay inside the series: no bound checks
        const int64_t tf = max(t0, min(t1, T - (int64_t)tau_max));
        const float2* row = S + t0 * P + p;
        int64_t t = t0;
        for (; t < tf; ++t, row += P) {
            const float2 a = row[0];
            add_mean(a);
#pragma unroll
            for (int k = 0; k < kIsfGroup; ++k) add(k, a, row[off[k]]);
        }
        for (; t < t1; ++t, row += P) {
            const float2 a = row[0];
            add_mean(a);
#pragma unroll
            for (int k = 0; k < kIsfGroup; ++k)
                if (k < nt && t + s_tau[k] < T) add(k, a, row[off[k]]);
        }
#pragma unroll
        for (int k = 0; k < kIsfGroup; ++k) {
            dre[k] += (double)are[k] - (double)cre[k];
            dim[k] += (double)aim[k] - (double)cim[k];
            are[k] = cre[k] = aim[k] = cim[k] = 0.0f;
        }
        dmean += (double)macc - (double)mcomp;
        macc = mcomp = 0.0f;
    }
    const double m = dmean / (double)T;  // F(q,0) sum f^2
#pragma unroll
    for (int k = 0; k < kIsfGroup; ++k) {
        if (k < nt) {
            const double n = (double)(T - s_tau[k]);
            const double re = dre[k] / n, im = dim[k] / n;
            const int64_t o = (int64_t)(g0 + k) * P + p;
            F[o] = make_double2(re * inv_sum_f2, im * inv_sum_f2);
            if (Fhat) Fhat[o] = make_double2(re / m, im / m);
        }
    }
}

// one thread per in-ring pixel (ring-major order); Ks sorted ascending, row
// k_row[i] of the output receives K = Ks[i]
__global__ void isf_contrast_kernel(const double2* __restrict__ Fhat, int64_t Kmax, int64_t P,
                                    const int32_t* __restrict__ perm, int64_t n_in,
                                    const int32_t* __restrict__ Ks, const int32_t* __restrict__ k_row, int n_K,
                                    double* __restrict__ b) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_in) return;
    const int64_t p = perm[q];
    double A = 0.0, B = 0.0;  // sums over d in [1, K) of |F_hat(d)|^2 and d |F_hat(d)|^2
    int i = 0;
    for (int64_t d = 1; d <= Kmax && i < n_K; ++d) {
        while (i < n_K && Ks[i] == d) {
            const double K = (double)d;
            b[(int64_t)k_row[i] * n_in + q] = (K + 2.0 * (K * A - B)) / (K * K);
            ++i;
        }
        if (d == Kmax) break;
        const double2 z = Fhat[d * P + p];
        const double a = fma(z.x, z.x, z.y * z.y);
        A += a;
        B = fma((double)d, a, B);
    }
}

// one warp per (K, ring): mean of b over the ring's pixels, fixed order
__global__ void ring_mean_kernel(const double* __restrict__ b, int64_t n_in, const int64_t* __restrict__ ring_start,
                                 int n_rings, int n_K, double* __restrict__ out) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= (int64_t)n_K * n_rings) return;
    const int ik = (int)(i / n_rings);
    const int r = (int)(i - (int64_t)ik * n_rings);
    const int64_t a0 = ring_start[r], a1 = ring_start[r + 1];
    if (a1 == a0) {
        if (lane == 0) out[i] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
        return;
    }
    const double* row = b + (int64_t)ik * n_in;
    double acc = 0.0;
    for (int64_t a = a0 + lane; a < a1; a += 32) acc += row[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = acc / (double)(a1 - a0);
}

// The prefix runs over frame segments in parallel (one thread per in-ring
// pixel alone is too few to hide the load latency): segment_total_kernel sums
// each (pixel, segment), then prefix_kernel starts every segment from the sum
// of the totals before it.  The totals sit in kPrefixSegs rows after C's T+1.
constexpr int kAhead = 8;  // frames' loads in flight per thread

__device__ __forceinline__ double sum_frames(const float* __restrict__ I, int64_t P, int64_t p, int64_t t0,
                                             int64_t t1, double acc, double* __restrict__ C, int64_t n_in,
                                             int64_t q) {
    int64_t t = t0;
    for (; t + kAhead <= t1; t += kAhead) {
        float x[kAhead];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) x[k] = I[(t + k) * P + p];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            acc += (double)x[k];
            if (C) C[(t + k + 1) * n_in + q] = acc;
        }
    }
    for (; t < t1; ++t) {
        acc += (double)I[t * P + p];
        if (C) C[(t + 1) * n_in + q] = acc;
    }
    return acc;
}

// grid (pixel blocks, segments): tot[s][q] = sum of I over segment s
__global__ void segment_total_kernel(const float* __restrict__ I, int64_t T, int64_t P,
                                     const int32_t* __restrict__ perm, int64_t n_in, int64_t seg_len,
                                     double* __restrict__ tot) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_in) return;
    const int64_t s = blockIdx.y;
    const int64_t t0 = s * seg_len, t1 = min(T, t0 + seg_len);
    tot[s * n_in + q] = sum_frames(I, P, perm[q], t0, t1, 0.0, nullptr, n_in, q);
}

// grid (pixel blocks, segments): C[t+1][q] for the frames t of segment s
__global__ void prefix_kernel(const float* __restrict__ I, int64_t T, int64_t P,
                              const int32_t* __restrict__ perm, int64_t n_in, int64_t seg_len,
                              const double* __restrict__ tot, double* __restrict__ C) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_in) return;
    const int64_t s = blockIdx.y;
    double acc = 0.0;
    for (int64_t k = 0; k < s; ++k) acc += tot[k * n_in + q];
    if (s == 0) C[q] = 0.0;
    const int64_t t0 = s * seg_len, t1 = min(T, t0 + seg_len);
    sum_frames(I, P, perm[q], t0, t1, acc, C, n_in, q);
}

// block = one chunk (ring, start, count) and a slice of `kw_slice` entries of
// the (K,w) list; its warps stride over the slice
// One warp takes 8 consecutive (K, w) entries: every lane sums x and x^2 over
// its pixels of the chunk for all 8, then one transposed butterfly reduces
// the 8 pairs together (lanes split the values in half at offsets 16, 8 and
// 4, then add at 2 and 1), 9 FP64 additions per lane and sum instead of 40;
// the kernel is bound by the FP64 pipe.  Lane 4j holds the totals of entry j.
constexpr int kKwGroup = 8;

__device__ __forceinline__ double halve(double* v, int n, int lane, int off) {
    // v[0 .. 2n) -> v[0 .. n): lanes with the `off` bit keep the upper half
    const bool up = (lane & off) != 0;
    for (int k = 0; k < n; ++k) {
        const double send = up ? v[k] : v[k + n];
        const double keep = up ? v[k + n] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
    return v[0];
}

__global__ void window_kernel(const double* __restrict__ C, int64_t n_in, const int4* __restrict__ chunks,
                              int n_chunks, const int32_t* __restrict__ Ks, const int64_t* __restrict__ kw_off,
                              int n_K, int64_t n_kw, int64_t kw_slice, double2* __restrict__ partial) {
    const int4 ch = chunks[blockIdx.x];  // (ring, start, count, 0)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t kw0 = (int64_t)blockIdx.y * kw_slice;
    const int64_t kw1 = min(n_kw, kw0 + kw_slice);
    int ik = 0;
    for (int64_t base = kw0 + (int64_t)warp * kKwGroup; base < kw1; base += (int64_t)nwarps * kKwGroup) {
        double s1[kKwGroup], s2[kKwGroup];
#pragma unroll
        for (int j = 0; j < kKwGroup; ++j) {
            s1[j] = s2[j] = 0.0;
            const int64_t kw = base + j;
            if (kw >= kw1) continue;
            while (ik + 1 < n_K && kw >= kw_off[ik + 1]) ++ik;
            while (ik > 0 && kw < kw_off[ik]) --ik;
            const int64_t K = Ks[ik];
            const int64_t w = kw - kw_off[ik];
            const double* c0 = C + (w * K) * n_in;
            const double* c1 = C + ((w + 1) * K) * n_in;
            for (int i = lane; i < ch.z; i += 32) {
                const int64_t q = ch.y + i;
                const double x = c1[q] - c0[q];
                s1[j] += x;
                s2[j] = fma(x, x, s2[j]);
            }
        }
        halve(s1, 4, lane, 16);
        halve(s1, 2, lane, 8);
        double t1 = halve(s1, 1, lane, 4);
        halve(s2, 4, lane, 16);
        halve(s2, 2, lane, 8);
        double t2 = halve(s2, 1, lane, 4);
        t1 += __shfl_xor_sync(0xffffffffu, t1, 2);
        t2 += __shfl_xor_sync(0xffffffffu, t2, 2);
        t1 += __shfl_xor_sync(0xffffffffu, t1, 1);
        t2 += __shfl_xor_sync(0xffffffffu, t2, 1);
        // lane bits 16, 8, 4 chose the upper halves: entry j = 4 b16 + 2 b8 + b4
        const int j = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        const int64_t kw = base + j;
        if ((lane & 3) == 0 && kw < kw1) partial[kw * n_chunks + blockIdx.x] = make_double2(t1, t2);
    }
}

// one warp per ((K,w), ring): the ring's chunk partials added in chunk order
__global__ void ring_sums_kernel(const double2* __restrict__ partial, int n_chunks, int64_t n_kw,
                                 const int32_t* __restrict__ ring_first_chunk, int n_rings, double2* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_kw * n_rings) return;
    const int64_t kw = i / n_rings;
    const int r = (int)(i - kw * n_rings);
    const double2* row = partial + kw * n_chunks;
    double s1 = 0.0, s2 = 0.0;
    for (int c = ring_first_chunk[r]; c < ring_first_chunk[r + 1]; ++c) {
        s1 += row[c].x;
        s2 += row[c].y;
    }
    out[i] = make_double2(s1, s2);
}

// one warp per (K, ring): lanes take windows w = lane, lane + 32, ...; the
// per-lane sums of beta_w are reduced by a fixed shuffle tree (deterministic)
__global__ void finalize_kernel(const double2* __restrict__ partial, int n_chunks,
                                const int32_t* __restrict__ Ks, const int64_t* __restrict__ kw_off, int n_K,
                                int64_t T, const int32_t* __restrict__ ring_first_chunk,
                                const int32_t* __restrict__ ring_count, int n_rings, double* __restrict__ beta) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= (int64_t)n_K * n_rings) return;
    const int ik = (int)(i / n_rings);
    const int r = (int)(i - (int64_t)ik * n_rings);
    const int n = ring_count[r];
    if (n == 0) {
        if (lane == 0) beta[i] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
        return;
    }
    const int c0 = ring_first_chunk[r], c1 = ring_first_chunk[r + 1];
    const int64_t K = Ks[ik];
    const int64_t W = T / K;
    double acc = 0.0;
    for (int64_t w = lane; w < W; w += 32) {
        const double2* row = partial + (kw_off[ik] + w) * n_chunks;
        double s1 = 0.0, s2 = 0.0;
        for (int c = c0; c < c1; ++c) {
            s1 += row[c].x;
            s2 += row[c].y;
        }
        const double m1 = s1 / n, m2 = s2 / n;
        acc += (m2 - m1 * m1) / (m1 * m1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) beta[i] = acc / (double)W;
}

}  // namespace

int64_t xsvs_prefix_rows(int64_t T) { return T + 1 + kPrefixSegs; }

// C [T+1][n_in] prefix sums of the permuted pixels; the kPrefixSegs rows after
// them hold the segment totals
static cudaError_t launch_prefix(const float* I, int64_t T, int64_t P, const int32_t* d_perm, int64_t n_in,
                                 double* C, cudaStream_t st) {
    const int64_t segs = std::max<int64_t>(1, std::min<int64_t>(kPrefixSegs, T / 64));
    const int64_t seg_len = T > 0 ? (T + segs - 1) / segs : 1;
    double* tot = C + (T + 1) * n_in;
    const dim3 grid((unsigned)((n_in + 127) / 128), (unsigned)segs);
    if (segs > 1) {
        ++tl_kernel_launches;
        segment_total_kernel<<<grid, 128, 0, st>>>(I, T, P, d_perm, n_in, seg_len, tot);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    ++tl_kernel_launches;
    prefix_kernel<<<grid, 128, 0, st>>>(I, T, P, d_perm, n_in, seg_len, tot, C);
    return cudaGetLastError();
}

int g2_segments(int64_t T) {
    const int64_t blocks = (T + kFlush - 1) / kFlush;
    return (int)std::max<int64_t>(1, std::min<int64_t>(8, blocks));
}

size_t g2_workspace_bytes(int64_t T, int64_t P, int n_tau) {
    if (g2s_width(T) > 0) return 0;  // g2_series_kernel writes g2 directly
    return (size_t)g2_segments(T) * (size_t)(n_tau + 1) * (size_t)P * sizeof(double);
}

cudaError_t launch_g2(const float* I, int64_t T, int64_t P, const int32_t* d_taus, int n_tau,
                      double* g2, double* mean, void* ws, cudaStream_t st) {
    if (P == 0 || n_tau == 0) return cudaSuccess;
    // the series kernel where 16 or 32 pixels' series fit in shared memory;
    // 2 delays per thread on 16 pixels keep about 512 (pixel, delay group)
    // items per block
    const int W = g2s_width(T);
    if (W == 32) return launch_g2_series<4>(I, T, P, d_taus, n_tau, W, g2, mean, st);
    if (W == 16) return launch_g2_series<2>(I, T, P, d_taus, n_tau, W, g2, mean, st);
    const int n_seg = g2_segments(T);
    const int64_t blocks = (T + kFlush - 1) / kFlush;
    const int64_t seg_len = (blocks + n_seg - 1) / n_seg * kFlush;
    double* part = static_cast<double*>(ws);
    double* mpart = part + (size_t)n_seg * n_tau * P;
    dim3 grid((unsigned)((P + kG2Threads - 1) / kG2Threads), (unsigned)((n_tau + kTauGroup - 1) / kTauGroup),
              (unsigned)n_seg);
    ++tl_kernel_launches;
    g2_kernel<<<grid, kG2Threads, 0, st>>>(I, T, P, d_taus, n_tau, seg_len, part, mpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)n_tau * P;
    ++tl_kernel_launches;
    g2_finish_kernel<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(part, mpart, n_seg, T, P, d_taus, n_tau, g2,
                                                                       mean);
    return cudaGetLastError();
}

cudaError_t launch_xsvs_partial(const float* I, int64_t T, int64_t P, const int32_t* d_perm, const int4* d_chunks,
                               int n_chunks, int64_t n_in_rings, const int32_t* d_K, const int64_t* d_kw_off, int n_K,
                               int64_t n_kw, const int32_t* d_ring_first_chunk, int n_rings, double* prefix,
                               double2* partial, double* sums, cudaStream_t st) {
    if (n_in_rings > 0) {
        cudaError_t e = launch_prefix(I, T, P, d_perm, n_in_rings, prefix, st);
        if (e != cudaSuccess) return e;
        int64_t slice = 64;
        if ((n_kw + slice - 1) / slice > 65535) slice = (n_kw + 65534) / 65535;
        const dim3 wgrid((unsigned)n_chunks, (unsigned)std::max<int64_t>(1, (n_kw + slice - 1) / slice));
        ++tl_kernel_launches;
        window_kernel<<<wgrid, 256, 0, st>>>(prefix, n_in_rings, d_chunks, n_chunks, d_K, d_kw_off, n_K, n_kw, slice,
                                             partial);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t items = n_kw * n_rings;
    if (items == 0) return cudaSuccess;
    ++tl_kernel_launches;
    ring_sums_kernel<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(partial, n_chunks, n_kw, d_ring_first_chunk,
                                                                       n_rings, reinterpret_cast<double2*>(sums));
    return cudaGetLastError();
}

cudaError_t launch_isf(const float* amp, int64_t T, int64_t P, const int32_t* d_taus, int n_tau, double inv_sum_f2,
                       double* F, double* Fhat, cudaStream_t st) {
    if (P == 0 || n_tau == 0) return cudaSuccess;
    dim3 grid((unsigned)((P + kG2Threads - 1) / kG2Threads), (unsigned)((n_tau + kIsfGroup - 1) / kIsfGroup));
    ++tl_kernel_launches;
    isf_kernel<<<grid, kG2Threads, 0, st>>>(reinterpret_cast<const float2*>(amp), T, P, d_taus, n_tau, inv_sum_f2,
                                            reinterpret_cast<double2*>(F), reinterpret_cast<double2*>(Fhat));
    return cudaGetLastError();
}

cudaError_t launch_isf_contrast(const double* Fhat, int64_t Kmax, int64_t P, const int32_t* d_perm, int64_t n_in,
                                const int32_t* d_K_sorted, const int32_t* d_k_row, int n_K,
                                const int64_t* d_ring_start, int n_rings, double* b_pixel, double* out,
                                cudaStream_t st) {
    if (n_in > 0) {
        ++tl_kernel_launches;
        isf_contrast_kernel<<<(unsigned)((n_in + 127) / 128), 128, 0, st>>>(
            reinterpret_cast<const double2*>(Fhat), Kmax, P, d_perm, n_in, d_K_sorted, d_k_row, n_K, b_pixel);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t items = (int64_t)n_K * n_rings;
    ++tl_kernel_launches;
    ring_mean_kernel<<<(unsigned)((items * 32 + 127) / 128), 128, 0, st>>>(b_pixel, n_in, d_ring_start, n_rings,
                                                                         n_K, out);
    return cudaGetLastError();
}

cudaError_t launch_xsvs(const float* I, int64_t T, int64_t P, const int32_t* d_perm,
                        const int4* d_chunks, int n_chunks, int64_t n_in_rings,
                        const int32_t* d_K, const int64_t* d_kw_off, int n_K, int64_t n_kw,
                        const int32_t* d_ring_first_chunk, const int32_t* d_ring_count,
                        int n_rings, double* prefix, double2* partial, double* beta,
                        cudaStream_t st) {
    if (n_in_rings > 0) {
        cudaError_t e = launch_prefix(I, T, P, d_perm, n_in_rings, prefix, st);
        if (e != cudaSuccess) return e;
        // slices of the (K,w) list give enough blocks to keep the SMs busy
        int64_t slice = 64;
        if ((n_kw + slice - 1) / slice > 65535) slice = (n_kw + 65534) / 65535;
        const dim3 wgrid((unsigned)n_chunks, (unsigned)std::max<int64_t>(1, (n_kw + slice - 1) / slice));
        ++tl_kernel_launches;
        window_kernel<<<wgrid, 256, 0, st>>>(prefix, n_in_rings, d_chunks, n_chunks, d_K, d_kw_off, n_K, n_kw,
                                             slice, partial);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t items = (int64_t)n_K * n_rings;  // one warp each
    ++tl_kernel_launches;
    finalize_kernel<<<(unsigned)((items * 32 + 127) / 128), 128, 0, st>>>(partial, n_chunks, d_K, d_kw_off, n_K, T,
                                                                     d_ring_first_chunk, d_ring_count, n_rings, beta);
    return cudaGetLastError();
}

}  // namespace xs
