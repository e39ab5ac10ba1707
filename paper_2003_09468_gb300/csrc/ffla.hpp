// Double-float overlap, projection, inverse and log-determinant (ffla.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ffla {

// Bytes of the double-float overlap array Sff[WS][N][N] (float4 per complex entry).
size_t overlap_scratch_bytes(int WS, int N);

// S = A^dag phi per walker-spin into Sff (A block-diagonal: A[k][M][n], phi[WS][Nk*M][N]).
// With B (the trial projector A (A^dag A)^-1, [k][M][n]) also phi_perp = phi - B S in fp32
// and mx[ws] = max |phi_perp| (mx must hold zeros, or smaller maxima, on entry).
cudaError_t overlap(const zc* A, const zc* phi, const zc* B, float4* Sff, float2* phi_perp, unsigned long long* mx,
                    int WS, int nk, int M, int n, int N, cudaStream_t st);

// log det of every Sff matrix into logdet[WS] (sing[ws] = 1 and flags[0] incremented for a
// singular one).  With out != nullptr also S^-T as fp16 split planes out[WS][4][N][Np]
// with per-matrix scale s_out[ws].  Sff is overwritten.
cudaError_t invert(float4* Sff, int WS, int N, zc* logdet, int* sing, int* flags, __half* out, int Np, float* s_out,
                   cudaStream_t st);

}  // namespace ffla
