// Block preconditioner of the Schur complement M = J A^-1 S for the inner
// GMRES of the approximate Schur preconditioner (schur_block.cu).
#pragma once

#include <cuda_runtime.h>

namespace ibrd {

// Per blob up to kBlockMax slots: itself first, then its nearest neighbours
// within the cutoff. Model of M: a / r + c0 + c2 r^2 (r >= rmin) off the
// diagonal, diag on it.
constexpr int kBlockMax = 32;
struct BlockModel {
  float a, c0, c2, diag, rmin;
};

// The constant C of the zero-mean periodic Green's function of -Laplace in a
// box lx x ly x lz: G(r) = 1 / (4 pi r) + C + O(r^2) (Ewald sum, any shape).
double periodic_constant(double lx, double ly, double lz);

// Slots (idx, cnt) and rows (val) of P for n blobs at q (n x 3 FP64, any
// position; pos: n float4 of scratch).
void launch_block_setup(const double* q, int n, double lx, double ly, double lz, double cutoff, BlockModel mdl,
                        float4* pos, int* idx, int* cnt, float* val, cudaStream_t s);

// y = P (x - *shift) (shift nullable; y must not overlap x), and per-CTA sums
// of y in partial[0 .. kBlockApplyBlocks) (their total is sum(y)); with mean
// non-null also *mean = mean_scale * sum(y), formed by the launch's last CTA
// (ticket: a per-handle counter, 0 between uses).
constexpr int kBlockApplyBlocks = 608;
template <typename Tin, typename Tout>
void launch_block_apply(const int* idx, const int* cnt, const float* val, const Tin* x, const double* shift, int n,
                        Tout* y, double* partial, cudaStream_t s, unsigned* ticket = nullptr,
                        double* mean = nullptr, double mean_scale = 0.0);

}  // namespace ibrd
