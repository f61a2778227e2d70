// Per-chunk argument block shared by the per-batch kernels (decode, r x r
// systems, row operands, fused N-1, final reduction) and the status codes of
// a topology.
#pragma once

#include "internal.cuh"

namespace dcf {

enum : int { ST_OK = 0, ST_ISLAND = 1, ST_INVALID = 2 };

struct QInfo {
  int tau, r, ks, status;
};

struct GridDev {
  const int *f, *t;
  const double* b;
  const int *inc_ptr, *inc_list, *nidx;
  const uint8_t* split_ok;  // [V] substations the study may split
  const uint8_t* out_ok;    // [E] branches the study may take out (outage candidates)
  int V, E;
};

struct BatchDev {
  const int *split_ptr, *split_sub;
  const uint64_t* split_mask;
  const int *out_ptr, *out_branch;
};

struct Args {
  // study
  int M, C, NN, T, U;
  int Mpad, ldc;  // padded monitored count (row stride of the per-row arrays), Phi[mon, cont] row stride
  const int *monN, *contN, *cpos, *mpos;
  const int* cont_pos;  // internal contingency index -> caller's position (outputs)
  const double *inv_lim, *PhiN, *bN;  // bN: susceptance of every needed branch
  const void* PhiMC;
  const double* p0;  // [NN][T]
  double tol;
  // chunk
  int nq;
  QInfo* qi;
  int* ent_n;
  int8_t* ent_s;
  double* ent_w;
  int16_t* mod_ptr;
  double *Kinv, *alpha, *Vt64;
  void *VtR, *Zs, *ptil, *rowmul, *diagv, *s;
  uint32_t* Zbf;  // BF16x3 form: Z / limit per monitored row as BF16 [hi KB | lo KB] (KB = 8 or 16), or null
  uint8_t* valid;
  int* nisl;
  void* pmax;
  int* parg;
  double* povl;
  void* p2max;  // second largest per-contingency maximum of each block (the tie band's check), or null
  int ncb;    // 64-contingency blocks of the N-1 kernels (the stride of their partial results)
  int C_eff;  // contingencies before the base-grid bridges (internal order)
  int c_rem;  // first contingency of a short remainder [c_rem, C_eff) left to the final pass
              // instead of an almost empty N-1 block (C_eff when there is none)
  const int* best_u;  // chosen injection candidate per (slot, timestep), or null
  // per (slot, timestep, internal contingency) maximum loading in the working
  // precision, -1 where skipped (read by the final pass's tie band), or null
  void* cmr;
  double tie_eps;       // tie band of the reported indices: eps * max(best, 1)
  const int* cont_inv;  // caller's position -> internal contingency
  // per (slot, timestep, internal contingency) below c_rem: the 16-row tile holding
  // the maximum (written by the tracking N-1 pass for the top-k cases), or null
  uint16_t* tile;
  int* err;  // set to 1 by a kernel whose bounded wait expired
  // outputs
  dcflow_results out;
};

}  // namespace dcf
