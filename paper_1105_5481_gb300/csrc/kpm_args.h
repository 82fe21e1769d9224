// Arguments of the device kernels: the scaled operator, the per-call
// parameters kept in device memory, and the arguments of one fused step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kpm {

// ----------------------------------------------------------------- operator descriptions
// Scaled operator applied by the fused step:  (S x)_i = d_i x_i + sum_j h_ij x_j
// where S = scale * (H - shift) (scale = 2/a, shift = b for the KPM step;
// scale = 1, shift = 0 for the Lanczos product).
struct ScalarBlock {        // written by the prescale kernel, read by every step
  double hu_re, hu_im;      // uniform scaled hopping -scale*t (stencil, hop == NULL)
  double du;                // uniform scaled diagonal -scale*shift (+ scale*0 onsite)
  float hu_re_f, hu_im_f, du_f, pad_f;
};

struct StencilGeom {
  int dims;
  int L[3];
  int stride[3];
  int periodic[3];
};

// Per-call parameters that live in device memory so that a captured graph
// can be replayed with new values.
struct RunParams {
  double a, b;              // rescaling of the current call
  unsigned long long seed;  // random-vector seed
  int s;                    // current realisation (advanced by the graph)
  int R;                    // vectors per realisation
  int S;
  int M;
  int flags;                // bit0: diverged
  int s0;                   // realisation index of s = 0 in the random-vector counters
};

// ----------------------------------------------------------------- kernel launchers
// Step modes
// MODE_DYN (device code only): MODE_FIRST or MODE_STEP chosen by a uniform
// runtime flag, so that a persistent kernel carries one copy of the traversal.
enum StepMode { MODE_FIRST = 0, MODE_STEP = 1, MODE_SPMV = 2, MODE_DYN = 3 };

struct StepArgs {
  // vectors: N x Rp (row-major, Rp contiguous), element T or complex<T>
  const void* x;     // v_n
  void* y;           // v_{n+1} (may alias w: written in place over v_{n-1})
  const void* w;     // v_{n-1} (MODE_STEP only)
  double* partial;   // [nCTA][2][Rp] for this step (NULL in MODE_SPMV)
  int64_t n;         // sites / rows
  int Rp;            // padded vector count
  int G;             // 16-byte chunks per row (row stride)
  int Gt;            // chunks per row handled by one CTA (G = Gt * gridDim.y)
  // operator
  const ScalarBlock* sc;
  const void* hs;    // stencil scaled hoppings [N][dims] (T or complex<T>), NULL => uniform
  const void* ds;    // stencil scaled diagonal [N] (T), NULL => uniform
  StencilGeom geom;
  const int64_t* rowptr;  // CSR
  const int32_t* col;     // CSR column indices, or ELL [n][ell_w]
  const void* vals;       // CSR / ELL scaled values (T or complex<T>)
  int ell_w;              // > 0: padded ELL rows of this width (col/vals are ELL)
  // Traversal.  The rows are visited in passes of Q = (threads / Gt) rows,
  // one row per thread group.  line_len == 0: pass P covers rows P*Q .. P*Q+Q-1
  // (natural order).  Otherwise pass P covers x = P % line_len on the Q
  // adjacent lattice lines (a line = the line_len sites sharing y, z)
  // (P / line_len)*Q .. +Q-1, so that the rows of one pass are each other's
  // y-neighbours.  CTAs take chunks of `chunk` consecutive passes in a
  // grid-stride loop, so all CTAs sweep one compact front of passes and every
  // neighbour row is reused within about one chunk round.
  int line_len;
  int lines;
  int line_L1;            // L[1] (3D: line -> y = line % L1, z = line / L1)
  int64_t passes;         // total passes
  int chunk;              // passes per chunk
  // 1: the chunks are taken from the last one down.  Consecutive steps of a
  // single solve alternate, so that a step starts on the rows the previous
  // step touched last, which are still in L2 (both vector blocks of a step
  // are re-read by the next one).  The batched kernel keeps one direction:
  // there a CTA's own rows of the previous step are still in its L1.
  int reverse;
  // TMA-fed padded-ELL step (FP32 vectors, MODE_STEP): shared-memory stages,
  // passes per tile, minimum CTAs per SM of the variant; tma_stages = 0: the
  // plain step
  int tma_stages;
  int tma_passes;
  int tma_minb;
  int tma_prefetch;       // >= 0: L2 prefetch of the off-tile neighbour rows of the tile
                          // that many tiles ahead; < 0: none
  int tma_stall;          // testing aid: the producer issues no copy (the waits run out)
  int* err;               // bit 2 set by a bounded wait that ran out (may be NULL)
};

struct LaunchCfg {
  int block;
  int grid;
};

}  // namespace kpm
