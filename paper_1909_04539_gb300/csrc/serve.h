// Work list of the grouped persistent solve used by the request server.
#pragma once

#include <stdint.h>

namespace bs {

enum { SERVE_F64 = 0, SERVE_F32_REFINE = 1 };

// One request of a batch, as the grouped kernel sees it.
struct GReq {
  const double* c64;  // primal sweep coefficients, FP64 (C_COUNT * N)
  const float* c32;   // primal sweep coefficients, FP32
  const float* lu_hi; // primal sweep coefficients s, l1, l2, u1, u2: FP32 high parts (5 * N)
  const float* lu_lo; //   ... low parts
  const float* dfrec; // primal coefficient pairs (SweepPlan::dfrec)
  void* B;            // SERVE_F64: double, solved in place; SERVE_F32_REFINE: float input
  double* X;          // SERVE_F32_REFINE: FP64 output (SERVE_F64: equals B)
  int64_t M;
  int N, width, mode;
  int pairs;          // SERVE_F64 in FP32 pairs (as bs_solve takes it for this handle)
};

// 32 consecutive systems of one request: one warp's work item.
struct GTile {
  int req;
  int j0;
};

struct GHeader {
  int n_req, n_tiles, pad0, pad1;
};

constexpr int kGroupMaxReq = 512;
constexpr int kGroupMaxTiles = 16384;
constexpr size_t kGroupReqOff = sizeof(GHeader);
constexpr size_t kGroupTileOff = kGroupReqOff + sizeof(GReq) * kGroupMaxReq;
constexpr size_t kGroupWorkBytes = kGroupTileOff + sizeof(GTile) * kGroupMaxTiles;

// Enqueue the grouped kernel on `st`, reading its work list from d_work.
cudaError_t launch_grouped(const unsigned char* d_work, int grid, cudaStream_t st);
int grouped_grid();

}  // namespace bs
