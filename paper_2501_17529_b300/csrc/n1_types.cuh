// Types and tile constants shared by the fused N-1 kernels and the host code
// that launches them (tensor maps, selected-contingency lists).
#pragma once

#include <cuda.h>

namespace dcf {

constexpr int kLT = 16;     // monitored rows per tile
constexpr int kCB = 64;     // contingencies per block
constexpr int kPhW = kCB + 4;  // tensor-core build: width of the TMA'd Phi tile and pitch (pairs) of the built tile
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bounded mbarrier wait

// Tensor maps of one N-1 pass: Phi[mon, cont] / limit (per study), Z^T / limit,
// p_f^T / limit and the metadata rows (per chunk of topologies).
struct N1Maps {
  CUtensorMap phi, zt, pt, meta;
};

// Selected-contingency mode: where the gathered Phi tile comes from.
struct SelArgs {
  const float* phicm;  // [C][mp] Phi[mon, cont] / limit transposed, zero rows mp > M
  int mp;
  const int* csel;     // [nq][C] selected internal contingencies, ascending
  const int* nsel;     // [nq]
  const int* work;     // [items] (topology << 6) | 64-contingency block, or null: block (cb, q) of the grid
};
constexpr int kPP = 20;  // pitch (floats) of a gathered Phi column: 16 rows + bank spread

}  // namespace dcf
