// Standard (dense) representation of Sec. 2.2 on the k-point kernels.
//
// The two-body operator of Cholesky vectors L_g is 1/2 sum_g L_g L_g^dag (as one-body
// operators) plus the one-body v0.  Writing L_g = A_g - i B_g with the Hermitian
// A_g = (L_g + L_g^dag)/2 and B_g = i (L_g - L_g^dag)/2 gives
//   L_g L_g^dag = A_g^2 + B_g^2 + i [A_g, B_g],
// and the commutators sum to zero whenever the integrals are symmetric under the exchange
// of the two electrons (v_pqrs = v_qpsr), which holds for Coulomb integrals and for any
// vector set closed under the adjoint.  The potentials of Sec. 2.2 are then exactly
// v_{g+} = i A_g and v_{g-} = i B_g: a system of 2G Hermitian vectors at a single
// k-point (Q = 0 = -Q), where the k-point kernels apply unchanged.  Real symmetric vectors
// (real orbitals at the Gamma point) have B_g = 0 and keep G vectors.
#include "dense.hpp"

namespace dense {
namespace {

__global__ void hermitian_vectors_kernel(const zc* L, zc* out, int G, int M, int hermitian) {
  const size_t per = (size_t)M * M, total = (size_t)G * per;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t g = e / per, pr = e % per;
    const int p = (int)(pr / M), r = (int)(pr % M);
    const zc a = L[e], b = L[g * per + (size_t)r * M + p];   // L_pr, L_rp
    const zc bc = zconj(b);
    out[e] = zscale(zadd(a, bc), 0.5);
    if (!hermitian) {
      const zc d = zsub(a, bc);                                  // (L - L^dag)_pr
      out[(G + g) * per + pr] = zmake(-0.5 * d.y, 0.5 * d.x);     // i d / 2
    }
  }
}

}  // namespace

cudaError_t hermitian_vectors(const zc* L, zc* out, int G, int M, int hermitian, cudaStream_t st) {
  const size_t total = (size_t)G * M * M;
  const unsigned blocks = (unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  hermitian_vectors_kernel<<<blocks, 256, 0, st>>>(L, out, G, M, hermitian);
  return cudaGetLastError();
}

}  // namespace dense
