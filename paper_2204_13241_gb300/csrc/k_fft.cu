// The FFT-based method of the paper (Sec. 3.2, Algorithm 2), written here as a
// cross-check of the direct method, not as its hot path:
//   spread_kernel    each atom adds f_i g_x g_y g_z (1D Gaussian weights on
//                    the k_a grid points nearest it, periodic) into a complex
//                    FP64 grid with atomics
//   fft_lines_kernel radix-2 decimation-in-time FFT of a group of grid lines
//                    per block in shared memory, run once per axis, FP64,
//                    coalesced; the n/2 twiddles exp(-2 pi i m / n) are built
//                    once per block with sincospi (GB300's FP64 pipe is
//                    narrow: a sincospi per butterfly had cost ten times the
//                    butterflies themselves), and the first two stages, whose
//                    twiddles are 1 and -i, multiply nothing
//   fft_gather_kernel P(n) / (G_x(n_x) G_y(n_y) G_z(n_z)) at the requested
//                    Miller indices, with G_a the 1D DFT of the truncated
//                    Gaussian centred at the origin (the transform of one
//                    Gaussian, Algorithm 2's f^eta, is a product of three);
//                    I = |.|^2 and the amplitude in the exp(+i q.r) sign.
// The normalisation of the Gaussian and the volume per grid point cancel in
// the division and are left out.  The path runs in FP64: dividing by the
// Gaussian's transform (e^{-q^2 eta^2 / 2}) amplifies rounding at large q, and
// a cross-check should show the method's own errors, not FP32 noise.
#include <cmath>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kMaxCut = 64;

__global__ void spread_kernel(const float* __restrict__ pos, const float* __restrict__ f, int64_t n_atoms,
                              FftGrid fg, double2* __restrict__ grid, int* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_atoms) return;
    const int n = fg.n;
    double w[3][kMaxCut];
    int first[3];
    bool ok = isfinite(f[i]);
    for (int a = 0; a < 3; ++a) {
        const double x = (double)pos[3 * i + a];
        ok = ok && isfinite(x) && fabs(x) < 1.0e6 * fg.h[a] * n;
        // the k grid points nearest x: indices ceil(x/h - k/2) + j
        const double u = x / fg.h[a];
        const double s0 = ceil(u - 0.5 * fg.k[a]);
        const double frac = u - s0;  // in [k/2 - 1, k/2]: small, exact enough in FP64
        first[a] = (int)(((int64_t)s0 % n + n) % n);
        for (int j = 0; j < fg.k[a]; ++j) {
            const double d = ((double)j - frac) * fg.h[a];
            w[a][j] = exp(-d * d * fg.inv_2eta2);
        }
    }
    if (!ok) {
        set_dev_error(err, kDevErrNonFinite);
        return;
    }
    const double fi = (double)f[i];
    for (int jz = 0; jz < fg.k[2]; ++jz) {
        const int iz = (first[2] + jz) % n;
        for (int jy = 0; jy < fg.k[1]; ++jy) {
            const int iy = (first[1] + jy) % n;
            const double wyz = fi * w[1][jy] * w[2][jz];
            double2* row = grid + ((int64_t)iz * n + iy) * n;
            for (int jx = 0; jx < fg.k[0]; ++jx) atomicAdd(&row[(first[0] + jx) % n].x, wyz * w[0][jx]);
        }
    }
}

// one block per `lb` lines; lines are indexed by L in [0, n^2): element j of
// line L sits at (L / n) * s_hi + (L % n) * s_lo + j * s_el.  Along x (s_el =
// 1) a line is contiguous and threads walk j; along y and z consecutive lines
// are consecutive x (s_lo = 1) and threads walk the lines, so the loads and
// stores are coalesced either way.  Shared memory: [lb][n] values, then the
// n/2 twiddles.
__global__ void fft_lines_kernel(double2* __restrict__ data, int n, int log2n, int lb, int64_t s_el, int64_t s_lo,
                                 int64_t s_hi) {
    extern __shared__ double2 buf[];
    double2* tw = buf + (size_t)lb * n;
    const int half_n = n >> 1;
    for (int m = threadIdx.x; m < half_n; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)n, &s, &c);
        tw[m] = make_double2(c, s);
    }
    const int64_t L0 = (int64_t)blockIdx.x * lb;
    const bool j_fast = s_el == 1;
    const int total = lb * n;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = j_fast ? idx / n : idx % lb;
        const int j = j_fast ? idx % n : idx / lb;
        const int64_t L = L0 + l;
        const double2* line = data + (L / n) * s_hi + (L % n) * s_lo;
        const int r = (int)(__brev((unsigned)j) >> (32 - log2n));
        buf[l * n + r] = line[(int64_t)j * s_el];
    }
    __syncthreads();
    for (int len = 2, tw_step = half_n; len <= n; len <<= 1, tw_step >>= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < lb * half_n; t += blockDim.x) {
            const int l = t / half_n, bt = t - l * half_n;
            const int pos = bt & (half - 1);
            const int i0 = l * n + (bt / half) * len + pos, i1 = i0 + half;
            const double2 u = buf[i0], v = buf[i1];
            double2 vw;
            if (len == 2) {
                vw = v;
            } else if (len == 4) {  // twiddles 1 and exp(-i pi / 2) = -i
                vw = pos ? make_double2(v.y, -v.x) : v;
            } else {
                const double2 w = tw[pos * tw_step];
                vw = make_double2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
            }
            buf[i0] = make_double2(u.x + vw.x, u.y + vw.y);
            buf[i1] = make_double2(u.x - vw.x, u.y - vw.y);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = j_fast ? idx / n : idx % lb;
        const int j = j_fast ? idx % n : idx / lb;
        const int64_t L = L0 + l;
        double2* line = data + (L / n) * s_hi + (L % n) * s_lo;
        line[(int64_t)j * s_el] = buf[l * n + j];
    }
}

__global__ void fft_gather_kernel(const double2* __restrict__ grid, int n, GridDesc g, const double2* __restrict__ G,
                                  float* __restrict__ I, float* __restrict__ amp) {
    const int64_t P = g.pixels();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int iz = (int)(p / plane);
    const int64_t rem = p - (int64_t)iz * plane;
    const int iy = (int)(rem / g.nx);
    const int ix = (int)(rem - (int64_t)iy * g.nx);
    const int mx = ((g.nx0 + ix) % n + n) % n, my = ((g.ny0 + iy) % n + n) % n, mz = ((g.nz0 + iz) % n + n) % n;
    const double2 v = grid[((int64_t)mz * n + my) * n + mx];
    // G = G_x G_y G_z
    const double2 gx = G[mx], gy = G[n + my], gz = G[2 * n + mz];
    const double2 gxy = make_double2(gx.x * gy.x - gx.y * gy.y, gx.x * gy.y + gx.y * gy.x);
    const double2 gg = make_double2(gxy.x * gz.x - gxy.y * gz.y, gxy.x * gz.y + gxy.y * gz.x);
    const double den = gg.x * gg.x + gg.y * gg.y;
    // P / G = P conj(G) / |G|^2 is p^e (exp(-i q.r)); the amplitude here is its conjugate
    const double re = (v.x * gg.x + v.y * gg.y) / den;
    const double im = (v.y * gg.x - v.x * gg.y) / den;
    I[p] = (float)(re * re + im * im);
    if (amp) {
        amp[2 * p] = (float)re;
        amp[2 * p + 1] = (float)(-im);
    }
}

}  // namespace

cudaError_t launch_fft_frame(const float* pos, const float* f, int64_t n_atoms, const FftGrid& fg, double2* grid,
                             const GridDesc& g, const double2* d_G, float* I, float* amp, int* err, cudaStream_t st) {
    const int n = fg.n;
    if (fg.k[0] > kMaxCut || fg.k[1] > kMaxCut || fg.k[2] > kMaxCut) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(grid, 0, (size_t)n * n * n * sizeof(double2), st);
    if (e != cudaSuccess) return e;
    if (n_atoms > 0) {
        ++tl_kernel_launches;
        spread_kernel<<<(unsigned)((n_atoms + 127) / 128), 128, 0, st>>>(pos, f, n_atoms, fg, grid, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    // lines per block: 64 KB of values (lb divides n, both powers of two) plus
    // the twiddles
    const int lb = std::max(1, std::min(n, 4096 / n));
    const int threads = 512;
    const size_t smem = ((size_t)lb * n + n / 2) * sizeof(double2);
    e = cudaFuncSetAttribute((const void*)fft_lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    // x lines (stride 1), then y (stride n), then z (stride n^2)
    const int64_t strides[3][3] = {{1, n, nn}, {n, 1, nn}, {nn, 1, n}};
    for (int a = 0; a < 3; ++a) {
        ++tl_kernel_launches;
        fft_lines_kernel<<<(unsigned)(nn / lb), threads, smem, st>>>(grid, n, log2n, lb, strides[a][0],
                                                                     strides[a][1], strides[a][2]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t P = g.pixels();
    if (P == 0) return cudaSuccess;
    ++tl_kernel_launches;
    fft_gather_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(grid, n, g, d_G, I, amp);
    return cudaGetLastError();
}

}  // namespace xs
