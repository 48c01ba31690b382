// Fused (single cooperative launch) PCG for one AMEn local system.
#pragma once
#include "common.cuh"

namespace ttiga {

template <typename T> struct PcgArgs {
  const T *PhiL;  // [rl][Rl][rl]
  const T *PhiR;  // [rr][Rr][rr]
  const T *A;     // [Rl][n][2p+1][Rr]
  const float *Lf;  // band Cholesky factors [n][p+1][rl*rr] (FP32; reciprocal diagonal in slot p)
  // block-band preconditioner (edge != 0), block size bbM, bbS super-rows of q = p bbM:
  // the odd-even reduction factors Linv, Ul, Ur [bbS][q][q] (FP32, see bbprec.cuh)
  const float *bbLinv, *bbUl, *bbUr;
  int edge, bbM, bbS;
  const T *b;     // right-hand side [rl][n][rr]
  T *x, *r, *z, *pv, *pv2, *q;  // solution and work vectors [rl][n][rr] (pv, pv2: p double buffer)
  // per-CTA slab scratch of the dense phase, grid x dense_stride, used when dense_off < 0:
  // p [rl][S+2p][rr], T1 [rl][S+2p][rr][Rr], T2 [Rl][rl][S][rr] back to back
  T *scratch;
  double *part;   // 3 * grid partial sums
  struct Barrier *bar;
  int *err;       // set to 1 when a grid barrier wait runs out
  double *out;    // [0] iterations, [1] final ||r||^2
  unsigned long long *trace;  // optional phase timestamps of CTA 0 (null: off)
  int trace_cap;
  int rl, rr, Rl, Rr, n, p;
  double tol2;    // stop when ||b - B x||^2 <= tol2
  int maxit;
  int slots;      // band systems staged per CTA at a time (set by pcg_fused_grid)
  int resident;   // 1: every band system has its own slot, factors gathered once (set by pcg_fused_grid)
  int slab;       // mode rows per slab of the dense phase (set by pcg_fused_grid)
  long long p_stride, t1_stride, t2_stride, dense_stride;  // slab scratch sizes in elements (set by pcg_fused_grid)
  int dense_off;  // byte offset of the slab scratch in dynamic shared memory, -1: in `scratch` (pcg_fused_grid)
  int iface_off;  // byte offset of PhiR, PhiL copies in dynamic shared memory, -1: read from global
  int phr_ld;     // row stride of the shared copy of PhiR (rr rounded up to odd)
  int smem;       // dynamic shared memory bytes (set by pcg_fused_grid)
  // Tensor-core stages (FP32 PCG only): set tc = 1 to ask for them; pcg_fused_grid
  // keeps it when the operands fit in shared memory and TMEM, else clears it.  The
  // right- and left-interface contractions then run as tcgen05 kind::tf32 MMAs with
  // the 3xTF32 split.  Padded shapes: stage A M = tcMA (Ps rows), N = tcNA (rr Rr),
  // K = tcKA (rr); stage C M = tcMC (S rr), N = tcNC (rl), K = tcKC (Rl rl).
  int tc;
  int tc_off;     // byte offset of the operands in dynamic shared memory
  int tc_cols;    // TMEM columns allocated per CTA
  int tcMA, tcNA, tcKA, tcMC, tcNC, tcKC;
};

// Number of CTAs for the cooperative launch (all co-resident).
template <typename T> int pcg_fused_grid(Ctx *c, PcgArgs<T> &a);
// Launch on the context stream; bar must hold 8 zeroed-or-stale bytes (reset here).
template <typename T> void pcg_fused(Ctx *c, PcgArgs<T> a, int grid);
// z = B^{-1} b with a built block-band preconditioner (one CTA, the E phase of PCG).
struct BBPrec;
template <typename T>
void bb_solve_once(Ctx *c, const BBPrec &P, int rl, int rr, int n, int p, const T *b, T *z);

}  // namespace ttiga
