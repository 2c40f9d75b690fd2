// On-chip interleaved sweep for FP32 arithmetic (FP32 or BF16 input, FP32
// output): the forward-sweep values of a tile of systems never leave shared
// memory, so HBM sees only the compulsory traffic (read B once, write X once).
//
// One CTA is one warp and owns a tile of T = 32 (or 16) neighbouring systems,
// one lane per system.  Shared memory holds the tile's whole N x T block.  At
// the start of a tile one lane requests every row chunk of B with 2D TMA
// loads (cp.async.bulk.tensor, box T x 32 rows), each chunk completing on its
// own mbarrier, so the whole tile is in flight at once.  The forward sweep
// walks the chunks as they land and overwrites B with the forward values in
// place; the backward sweep walks back and overwrites them with X; each
// finished chunk leaves by a TMA store.  Tiles are persistent per CTA; several
// one-warp CTAs share an SM, so one tile's loads overlap another's sweeps.
// Out-of-range columns and rows are zero-filled by the loads and clipped by
// the stores.  Every mbarrier wait is bounded: on time-out the kernel records
// an error code (read with bs_device_status), waits (bounded) for the copies
// it started, and returns.
#include <cuda.h>

#include <type_traits>

#include "sweep_kernels.cuh"

namespace bs {


constexpr int kTmaRows = 32;         // rows per chunk = box height
constexpr int kTmaU = 8;             // rows per register block (divides kTmaRows)
constexpr int kTmaMaxChunks = 128;   // N <= 4096
constexpr int kWaitSpins = 1 << 20;  // bounded mbarrier waits

__device__ int g_device_status = 0;

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity) {
  for (int it = 0; it < kWaitSpins; it++)
    if (mbar_try_wait(a, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* m, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* m, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   reinterpret_cast<uint64_t>(m)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

template <typename Sin>
__device__ __forceinline__ float widen(Sin v);
template <>
__device__ __forceinline__ float widen<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) {
  return bf16_bits_to_float(*reinterpret_cast<const unsigned short*>(&v));
}

// Shared memory: [coefficients (SMEM)] [d: Npad x T floats] [stage: Npad x T Sin, BF16 input only]
template <int BW, bool ADJ, bool SMEM, typename Sin, int T>
__global__ void __launch_bounds__(32)
k_sweep_tma(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout, Coefs<float> cf_g,
            int N, int64_t M, int ahead) {
  constexpr bool kStage = !std::is_same<Sin, float>::value;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[kTmaMaxChunks];
  const int lane = threadIdx.x;
  const int nch = (N + kTmaRows - 1) / kTmaRows;
  const int npad = nch * kTmaRows;
  const size_t cbytes = SMEM ? align_up((size_t)coef_arrays<BW>() * N * sizeof(float), 1024) : 0;
  const Coefs<float> cf = stage_coefs<BW, ADJ, SMEM>(cf_g, N, reinterpret_cast<float*>(smem));
  float* d = reinterpret_cast<float*>(smem + cbytes);
  Sin* stage = reinterpret_cast<Sin*>(smem + cbytes + (size_t)npad * T * sizeof(float));
  Sin* land = kStage ? stage : reinterpret_cast<Sin*>(d);
  const uint32_t mbar0 = smem_u32(&mbar[0]);
  if (lane == 0) {
    for (int c = 0; c < nch; c++) mbar_init(mbar0 + 8 * c, 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncwarp();
  const uint32_t chunk_in = (uint32_t)(kTmaRows * T * sizeof(Sin));
  const int64_t ntiles = (M + T - 1) / T;
  uint32_t parity = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, parity ^= 1u) {
    const int j0 = (int)(t * T);
    fence_proxy_async();  // earlier reads of this smem precede the async writes below
    __syncwarp();
    auto issue = [&](int c) {
      mbar_expect_tx(mbar0 + 8 * c, chunk_in);
      tma_load_2d(smem_u32(land + (size_t)c * kTmaRows * T), &tin, j0, c * kTmaRows, mbar0 + 8 * c);
    };
    if (lane == 0) {
      bulk_wait_read0();  // the previous tile's stores have read their rows
      for (int c = 0; c < nch && c < ahead; c++) issue(c);
    }
    __syncwarp();
    // forward sweep, chunk by chunk as the rows land
    float r1[1] = {0.f}, r2[1] = {0.f};
    int c = 0;
    for (; c < nch; c++) {
      if (lane == 0 && c + ahead < nch) issue(c + ahead);  // keep `ahead` chunks in flight
      const bool ok = mbar_wait_bounded(mbar0 + 8 * c, parity);
      if (!__all_sync(0xffffffffu, ok)) break;
      const int i0 = c * kTmaRows;
      const int rows = (N - i0) < kTmaRows ? (N - i0) : kTmaRows;
      if (lane < T) {
#pragma unroll 1
        for (int q0 = 0; q0 < rows; q0 += kTmaU) {
          const int n = (rows - q0) < kTmaU ? (rows - q0) : kTmaU;
          float f[kTmaU][1];
#pragma unroll
          for (int u = 0; u < kTmaU; u++) f[u][0] = widen<Sin>(land[(size_t)(i0 + q0 + u) * T + lane]);
          fwd_block<BW, ADJ, float, 1, kTmaU>(cf, i0 + q0, n, f, r1, r2);
#pragma unroll
          for (int u = 0; u < kTmaU; u++)
            if (u < n) d[(size_t)(i0 + q0 + u) * T + lane] = f[u][0];
        }
      }
    }
    if (c < nch) {  // a load never completed: record, drain what we started, leave
      if (lane == 0) {
        atomicExch(&g_device_status, 1);
        for (int q = c; q < nch && q < c + ahead + 1; q++) mbar_wait_bounded(mbar0 + 8 * q, parity);
        bulk_wait0();
      }
      __syncwarp();
      return;
    }
    // backward sweep; each finished chunk is stored
    r1[0] = r2[0] = 0.f;
    for (c = nch - 1; c >= 0; c--) {
      const int i0 = c * kTmaRows;
      const int rows = (N - i0) < kTmaRows ? (N - i0) : kTmaRows;
      if (lane < T) {
#pragma unroll 1
        for (int top = i0 + rows - 1; top >= i0; top -= kTmaU) {
          const int n = (top - i0 + 1) < kTmaU ? (top - i0 + 1) : kTmaU;
          float f[kTmaU][1];
#pragma unroll
          for (int u = 0; u < kTmaU; u++) f[u][0] = d[(size_t)(u < n ? top - u : top) * T + lane];
          bwd_block<BW, ADJ, float, 1, kTmaU>(cf, top, n, f, r1, r2);
#pragma unroll
          for (int u = 0; u < kTmaU; u++)
            if (u < n) d[(size_t)(top - u) * T + lane] = f[u][0];
        }
      }
      fence_proxy_async();  // make the writes visible to the store's async proxy
      __syncwarp();
      if (lane == 0) {
        tma_store_2d(&tout, j0, i0, smem_u32(d + (size_t)i0 * T));
        bulk_commit();
      }
    }
  }
  if (lane == 0) bulk_wait0();
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D map over an (N rows) x (M columns) row-major batch, box T x kTmaRows.
static bool make_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, size_t elem, int N, int64_t M, int T) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)M * elem};
  const cuuint32_t box[2] = {(cuuint32_t)T, (cuuint32_t)kTmaRows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Shared bytes of one CTA, or 0 if the tile does not fit.
static size_t tma_smem(int bw, int N, int T, size_t in_elem, bool smem_coefs) {
  const int npad = (N + kTmaRows - 1) / kTmaRows * kTmaRows;
  size_t b = smem_coefs ? align_up((size_t)(1 + 2 * bw) * N * sizeof(float), 1024) : 0;
  b += (size_t)npad * T * sizeof(float);
  if (in_elem != sizeof(float)) b += (size_t)npad * T * in_elem;
  return b;
}

template <int BW, bool ADJ, typename Sin>
static int try_launch(const SweepPlan& p, int N, const Sin* in, float* out, int64_t M, cudaStream_t st,
                      cudaError_t* err) {
  const DeviceInfo& di = device_info();
  if (N > kTmaMaxChunks * kTmaRows) return 0;
  const size_t per_sm = 227 * 1024;
  // pick the tile width and coefficient placement that give >= 3 CTAs per SM,
  // else >= 2, else fall back
  int T = 0;
  bool sc = false;
  size_t bytes = 0;
  for (int want = 3; want >= 2 && !T; want--)
    for (int tt : {32, 16})
      for (bool s : {true, false}) {
        if (T) break;
        const size_t b = tma_smem(BW, N, tt, sizeof(Sin), s);
        if ((b + 1024) * want <= per_sm && b <= (size_t)di.smem_optin) {
          T = tt;
          sc = s;
          bytes = b;
        }
      }
  if (!T) return 0;
  CUtensorMap mi, mo;
  const CUtensorMapDataType dti =
      std::is_same<Sin, float>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (!make_map(&mi, in, dti, sizeof(Sin), N, M, T)) return 0;
  if (!make_map(&mo, out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), N, M, T)) return 0;
  const Coefs<float> cf = coefs_of<float>(p.c32, N);
  int per = (int)(per_sm / (bytes + 1024));
  if (per > 32) per = 32;
  int64_t grid = (int64_t)di.sms * per;
  const int64_t tiles = (M + T - 1) / T;
  if (grid > tiles) grid = tiles;
  void (*k)(const CUtensorMap, const CUtensorMap, Coefs<float>, int, int64_t, int);
  if (T == 32)
    k = sc ? k_sweep_tma<BW, ADJ, true, Sin, 32> : k_sweep_tma<BW, ADJ, false, Sin, 32>;
  else
    k = sc ? k_sweep_tma<BW, ADJ, true, Sin, 16> : k_sweep_tma<BW, ADJ, false, Sin, 16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) {
    int ahead = (int)option(BS_OPT_TMA_AHEAD);
    if (ahead <= 0) ahead = 4;
    k<<<(int)grid, 32, bytes, st>>>(mi, mo, cf, N, M, ahead);
    e = cudaGetLastError();
  }
  *err = e;
  return 1;
}

// Returns 1 and sets *err if the on-chip kernel took the solve, 0 if the
// shape does not qualify (the caller then uses the streaming kernels).
// Conditions: interleaved layout, 16-byte aligned pointers, row pitch a
// multiple of 16 bytes for both tensors, and the tile fits shared memory.
template <typename Sin>
int sweep_tma(const SweepPlan& p, bool adjoint, int N, const Sin* in, float* out, int64_t M, cudaStream_t st,
              cudaError_t* err) {
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return 0;
  if ((M * (int64_t)sizeof(Sin)) % 16 || (M * 4) % 16) return 0;
  if (M > ((int64_t)1 << 31) - 64) return 0;
  if (p.bw == 1)
    return adjoint ? try_launch<1, true, Sin>(p, N, in, out, M, st, err)
                   : try_launch<1, false, Sin>(p, N, in, out, M, st, err);
  return adjoint ? try_launch<2, true, Sin>(p, N, in, out, M, st, err)
                 : try_launch<2, false, Sin>(p, N, in, out, M, st, err);
}

template int sweep_tma<float>(const SweepPlan&, bool, int, const float*, float*, int64_t, cudaStream_t, cudaError_t*);
template int sweep_tma<__nv_bfloat16>(const SweepPlan&, bool, int, const __nv_bfloat16*, float*, int64_t,
                                      cudaStream_t, cudaError_t*);

}  // namespace bs

extern "C" bs_status bs_device_status(int* code, int reset) {
  using namespace bs;
  if (!code) return set_error(BS_EINVAL, "bs_device_status: null output");
  cudaError_t e = cudaMemcpyFromSymbol(code, g_device_status, sizeof(int));
  if (e == cudaSuccess && reset) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
  }
  if (e != cudaSuccess) return cuda_error(e, "bs_device_status");
  return BS_OK;
}
