// Adjoint of the intensity with respect to atomic positions.
//
//   dL/dr_j = sum_q G_q 2 Re[conj(S_q) i q f_j e^{i q.r_j}]
//           = -2 f_j sum_q Im[H_q e^{i theta_qj}] q,          H_q = G_q conj(S_q)
// With q = 2 pi h^-T n and theta = 2 pi (n_x s_x + n_y s_y + n_z s_z):
//   dL/dr_j = -4 pi f_j h^-T Im[T_j],   T_j,a = sum_q n_a H_q e^{i theta_qj}.
// Because the phase factorises over the axes (Sec. 3.1, reciprocal-lattice q),
//   T_x = sum_{z,x} n_x E_xz Z,  T_y = sum_{z,x} E_xz Z_y,  T_z = sum_{z,x} n_z E_xz Z
// with Z(x,z) = sum_y H(x,y,z) E_y and Z_y(x,z) = sum_y n_y H(x,y,z) E_y:
// two complex contractions over n_y followed by per-atom sums over n_x, n_z.
//
// H is formed where it is used, by the kernel that writes the swizzled H image
// of the tensor-core contraction (k_adjoint_tc.cu); the contractions and the
// per-atom sums run there too.
#include "xs_internal.h"

namespace xs {

size_t adjoint_workspace_bytes(const GridDesc& g, int64_t n_pad) { return adjoint_tc_image_bytes(g, n_pad); }

cudaError_t launch_adjoint(const AtomRec* rec, int64_t n_atoms, int64_t n_pad, const GridDesc& g,
                           const Mat3& hinv, const float* amp, const float* dL_dI, void* workspace,
                           float* grad, int* err, int64_t timeout_ns, cudaStream_t st) {
    return launch_adjoint_tc(rec, n_atoms, n_pad, g, hinv, amp, dL_dI, workspace, grad, err, timeout_ns, st);
}

}  // namespace xs
