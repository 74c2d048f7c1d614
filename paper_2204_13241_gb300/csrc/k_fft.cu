// The FFT-based method of the paper (Sec. 3.2, Algorithm 2), written here as a
// cross-check of the direct method, not as its hot path:
//   spread_kernel    each atom adds f_i g_x g_y g_z (1D Gaussian weights on
//                    the k_a grid points nearest it, periodic) into a complex
//                    FP64 grid with atomics
//   fft_lines_kernel radix-2 decimation-in-time FFT of one grid line per
//                    block in shared memory (twiddles exp(-2 pi i j / len)
//                    from sincospi), run once per axis, FP64
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

// one block per line; lines are indexed by L in [0, n^2): element j of line L
// sits at (L / n) * s_hi + (L % n) * s_lo + j * s_el
__global__ void fft_lines_kernel(double2* __restrict__ data, int n, int log2n, int64_t s_el, int64_t s_lo,
                                 int64_t s_hi) {
    extern __shared__ double2 buf[];
    const int64_t L = blockIdx.x;
    double2* line = data + (L / n) * s_hi + (L % n) * s_lo;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int r = (int)(__brev((unsigned)j) >> (32 - log2n));
        buf[r] = line[(int64_t)j * s_el];
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
            const int pos = t & (half - 1);
            const int i0 = (t / half) * len + pos, i1 = i0 + half;
            double s, c;
            sincospi(-2.0 * (double)pos / (double)len, &s, &c);
            const double2 u = buf[i0], v = buf[i1];
            const double2 vw = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
            buf[i0] = make_double2(u.x + vw.x, u.y + vw.y);
            buf[i1] = make_double2(u.x - vw.x, u.y - vw.y);
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) line[(int64_t)j * s_el] = buf[j];
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
    const int threads = std::min(512, std::max(32, n / 2));
    const size_t smem = (size_t)n * sizeof(double2);
    const int64_t nn = (int64_t)n * n;
    // x lines (stride 1), then y (stride n), then z (stride n^2)
    const int64_t strides[3][3] = {{1, n, nn}, {n, 1, nn}, {nn, 1, n}};
    for (int a = 0; a < 3; ++a) {
        ++tl_kernel_launches;
        fft_lines_kernel<<<(unsigned)nn, threads, smem, st>>>(grid, n, log2n, strides[a][0], strides[a][1],
                                                              strides[a][2]);
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
