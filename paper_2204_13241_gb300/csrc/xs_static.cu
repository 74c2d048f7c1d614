// xs_intensity_fp32_static: the FP32 direct-sum intensity without any device
// allocation.
//
// Some callers cannot allocate device memory at the time they need an
// intensity: real-time or embedded hosts that fix their device memory budget
// at start-up, plug-ins running inside a host application that owns the
// device memory, and processes whose framework allocator already reserved the
// whole device.  This entry point serves them: its scratch (the phase records
// of every frame and the partial amplitudes of the atom splits) lives in one
// file-scope device array of kStaticScratchBytes that every GPU loading this
// library holds until the process exits.  The caller still passes inputs and
// outputs.
//
// The array's name is only a host-side stand-in in host code; its device
// address is looked up with cudaGetSymbolAddress, with the target device
// current, and passed to the kernels.  The lookup is repeated on every call: a
// cached address would go stale after cudaDeviceReset or in another context on
// the same device.  It enqueues no work; the first call on a device may load
// the library's device code there, so that first call should come before any
// stream capture.  All calls share the array and it keeps the last call's
// contents; every byte a call reads is written earlier in the same call, so
// nothing needs clearing.  Calls whose kernels overlap on the GPU (different
// streams without ordering) race on the array.
#include <cstdio>
#include <string>

#include "xs_api.h"
#include "xs_internal.h"

using namespace xs;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// the message is what xs_last_error() returns on the calling thread
xs_status static_fail(xs_status s, const std::string& msg) {
    set_last_error(msg.c_str());
    return s;
}

int64_t round_up64(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// true for device or managed memory (the kernels dereference the pointer)
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool invert3_static(const double* h, double* out) {
    const double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8], c02 = h[3] * h[7] - h[4] * h[6];
    const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (!(det != 0.0) || !(det == det) || det - det != 0.0) return false;
    out[0] = c00 / det;
    out[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    out[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    out[3] = c01 / det;
    out[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    out[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    out[6] = c02 / det;
    out[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    out[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    return true;
}

}  // namespace

extern "C" {

xs_status xs_intensity_fp32_static(const xs_traj* traj, const xs_qgrid* grid, float* I_out, float* amp_out,
                                   int* dev_err, void* cuda_stream) {
    if (!traj || !grid || !I_out) return static_fail(XS_ERR_INVALID_ARG, "trajectory, grid and I_out are required");
    if (grid->nx < 0 || grid->ny < 0 || grid->nz < 0) return static_fail(XS_ERR_INVALID_ARG, "negative grid extent");
    if (grid->nx > 65536 || grid->ny > 65536 || grid->nz > 65536)
        return static_fail(XS_ERR_INVALID_ARG, "grid extent too large");
    if (traj->n_atoms < 0 || traj->n_frames < 0) return static_fail(XS_ERR_INVALID_ARG, "negative atom or frame count");
    if (traj->n_atoms > (int64_t)1 << 31) return static_fail(XS_ERR_INVALID_ARG, "more than 2^31 atoms");
    if (traj->pos_on_host) return static_fail(XS_ERR_INVALID_ARG, "positions must be in device memory");
    if (traj->n_atoms > 0 && traj->n_frames > 0 && (!traj->pos || !traj->f))
        return static_fail(XS_ERR_INVALID_ARG, "positions or form factors are NULL");
    double hinv[9];
    if (!invert3_static(traj->box.h, hinv)) return static_fail(XS_ERR_INVALID_ARG, "singular or non-finite cell matrix");
    const GridDesc g{grid->nx0, grid->nx, grid->ny0, grid->ny, grid->nz0, grid->nz};
    const int64_t P = g.pixels(), T = traj->n_frames, N = traj->n_atoms;
    if (P == 0 || T == 0) return XS_OK;
    if (T > 65535) return static_fail(XS_ERR_INVALID_ARG, "more than 65,535 frames in one call");
    // every pointer a kernel dereferences must be device memory: a host
    // pointer is rejected here instead of faulting the GPU
    if (!on_device(I_out) || (amp_out && !on_device(amp_out)))
        return static_fail(XS_ERR_INVALID_ARG, "I_out and amp_out must be device memory");
    if (N > 0 && (!on_device(traj->pos) || !on_device(traj->f)))
        return static_fail(XS_ERR_INVALID_ARG, "positions and form factors must be device memory");
    if (dev_err && !on_device(dev_err)) return static_fail(XS_ERR_INVALID_ARG, "dev_err must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(XS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    int num_sms = 0;
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return static_fail(XS_ERR_CUDA, std::string("device attribute: ") + cudaGetErrorString(e));

    const int64_t n_pad = round_up64(N > 0 ? N : 1, 64);
    const DirectPlan plan = plan_direct(n_pad, T, g, num_sms);
    const size_t rec_bytes = (size_t)round_up64((int64_t)(T * n_pad * (int64_t)sizeof(AtomRec)), 256);
    const size_t need = rec_bytes + plan.partial_bytes;
    if (N > 0 && need > kStaticScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "xs_intensity_fp32_static needs %zu bytes of scratch for %lld frames x %lld atoms on %lld pixels; "
                 "its static scratch holds %zu bytes",
                 need, (long long)T, (long long)N, (long long)P, kStaticScratchBytes);
        return static_fail(XS_ERR_INVALID_ARG, buf);
    }

    // the array's address on the current device, looked up on every call
    // (no work is enqueued; a cached address could outlive its context)
    void* base = nullptr;
    e = cudaGetSymbolAddress(&base, g_static_scratch);
    if (e != cudaSuccess || !base)
        return static_fail(XS_ERR_CUDA,
                           std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));

    if (N == 0) {
        e = cudaMemsetAsync(I_out, 0, (size_t)T * P * sizeof(float), st);
        if (e == cudaSuccess && amp_out) e = cudaMemsetAsync(amp_out, 0, (size_t)T * P * 2 * sizeof(float), st);
        if (e != cudaSuccess) return static_fail(XS_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
        return XS_OK;
    }
    Mat3 hm;
    for (int i = 0; i < 9; ++i) hm.a[i] = hinv[i];
    PhaseOpts popt;
    popt.ortho = hinv[1] == 0.0 && hinv[2] == 0.0 && hinv[3] == 0.0 && hinv[5] == 0.0 && hinv[6] == 0.0 &&
                 hinv[7] == 0.0;
    popt.need_z = !(g.nz == 1 && g.nz0 == 0);
    popt.perm_mul = 1;
    AtomRec* rec = static_cast<AtomRec*>(base);
    void* partial = static_cast<unsigned char*>(base) + rec_bytes;
    e = launch_phase(traj->pos, traj->f, N, T, n_pad, hm, popt, rec, dev_err, st);
    if (e == cudaSuccess) e = launch_direct(rec, n_pad, T, g, plan, partial, I_out, amp_out, st);
    if (e != cudaSuccess) return static_fail(XS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return XS_OK;
}

}  // extern "C"
