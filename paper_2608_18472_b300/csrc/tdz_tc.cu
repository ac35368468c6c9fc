// Tensor-core axis transform of the fast-diagonalisation preconditioner (sm_103a: tiled TMA copies,
// tcgen05.mma of kind::tf32 with the accumulator in tensor memory).
//
// One transform contracts the fastest axis of a planar state with a dense per-axis matrix (Sec.
// "Eigenvalue problem": the S-orthonormal eigenvectors of the 1-D generalised problem T v = lam S v):
//
//   D(m, j) = sum_k (A_hi(m, k) + A_lo(m, k)) (B(j, k) + B_lo(j, k)),   m < rows, j < ncols, k < K,
//
// with A (rows x K) and B (ncols x K) row-major, k fastest: both operands are K-major. Each operand is
// a TF32 pair (hi = the value rounded to TF32, lo = the FP32 remainder; A is either given as a pair
// or given in FP32 and split in shared memory by the block), and the product keeps the
// three terms A_hi B_hi + A_lo B_hi + A_hi B_lo (the published "3xTF32" scheme, Ootomo and Yokota,
// 2022), so both operands enter with about 22 significant bits and the accumulation is FP32. Without
// B_lo (B exact in TF32) the third product is skipped.
//
// Row m of A is row r = m mod plane_rows of plane p = m / plane_rows; D is written with the new index
// slowest, out[p * plane_stride + j * plane_rows + r], so that after one transform per axis the axes
// are back in their original order. The result is written either as FP32 or again split into
// (hi, lo) TF32 terms for the next transform.
//
// One block computes a 128 x BN tile of D. Warp 0 issues the TMA copies of a ring of stages (A_hi,
// A_lo, B and B_lo, each 32 FP32 wide with the 128-byte swizzle), warp 1 allocates the accumulator
// columns in tensor memory and issues the MMAs (one thread), warps 2-5 read the accumulator back
// (tcgen05.ld, one lane per row) and store it. Every wait on an mbarrier gives up after about one
// second and raises the error word; the block then waits (bounded) for its own copies and MMAs and
// frees its tensor memory before it exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>

#include "tdz_arith.cuh"
#include "tdz_internal.h"

namespace tdz {
namespace tc {

constexpr int BM = 128;       // rows per tile: the M of one tcgen05.mma, one tensor-memory lane per row
constexpr int BK = 32;        // k per stage: 32 FP32 = 128 bytes, one 128-byte swizzle span
constexpr int UK = 8;         // k per tcgen05.mma of kind::tf32 (32 bytes)
constexpr int THREADS = 192;  // warp 0: copies, warp 1: MMAs, warps 2-5: accumulator read-back

// BLO: B is a TF32 pair too (a third product A_hi B_lo per k-step)
template <int BN, bool BLO>
struct Cfg {
  static constexpr uint32_t A_BYTES = BM * BK * 4;
  static constexpr uint32_t B_BYTES = BN * BK * 4;
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + (BLO ? 2 : 1) * B_BYTES;  // a multiple of 1024
  static constexpr int STAGES = (int)((192u * 1024u) / STAGE_BYTES);               // 2 to 4 stages
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;  // + slack to align the ring
};

// ---- PTX primitives
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr unsigned long long kLimitNs = 1000000000ull;  // one second per wait

// wait for the phase of the given parity; false once another role aborted or the limit passed
// (which aborts the block)
__device__ bool wait_phase(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtime_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtime_ns() - t0 > kLimitNs) {
      *abort_flag = 1;
      return false;
    }
  }
}
// the same wait, bounded by the time limit only (used on the way out)
__device__ bool wait_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtime_ns();
  while (!mbar_try_wait(bar, parity))
    if (gtime_ns() - t0 > kLimitNs) return false;
  return true;
}

// tiled 2-D TMA copy of one box at element coordinates (x = k, y = row); x is a multiple of 32
// FP32 = 128 bytes, so every copy starts on a 16-byte boundary
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// whole warp: allocate `ncols` tensor-memory columns (a power of two >= 32); the address goes to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor of a K-major tile stored with the 128-byte swizzle (rows of 128
// bytes, 8-row groups 1024 bytes apart): start address >> 4 in bits 0-13, leading-dimension offset
// (unused by this layout, 16 bytes) in bits 16-29, stride offset 1024 >> 4 in bits 32-45, the
// descriptor version 1 in bits 46-47 and the layout SWIZZLE_128B (2) in bits 61-63
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and 10-12 = 2),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// D (+)= A B^T on the tensor cores, issued by one thread; accumulate = 0 overwrites D
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive accumulator columns of this thread's lane (whole warp, lanes of its quadrant)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ASPLIT: A arrives as FP32 (one copy per stage, into the A_hi slot) and warps 2-5 split it in shared
// memory (hi in place, lo into the A_lo slot) before the MMAs read it; otherwise A arrives as a pair.
template <int BN, bool BLO, bool ASPLIT>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_axis(const __grid_constant__ CUtensorMap map_ahi, const __grid_constant__ CUtensorMap map_alo,
              const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_blo, long long rows,
              int K, int ncols, long long plane_rows, long long plane_stride, float* __restrict__ out_hi,
              float* __restrict__ out_lo, int* __restrict__ err) {
  using G = Cfg<BN, BLO>;
  constexpr int S = G::STAGES;
  constexpr uint32_t TX = G::STAGE_BYTES - (ASPLIT ? G::A_BYTES : 0u);  // bytes the copies of one stage bring
  extern __shared__ unsigned char dyn[];
  __shared__ __align__(8) uint64_t bars[3 * S + 1];  // full[S], empty[S], accumulator ready, split[S]
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const uint32_t ring = (smem_u32(dyn) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = (ncols + BN - 1) / BN;
  const int n0 = (int)(blockIdx.x % ntn) * BN;
  const long long m0 = (long long)(blockIdx.x / ntn) * BM;
  const int nk = (K + BK - 1) / BK;
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[S]), accum = smem_u32(&bars[2 * S]);
  const uint32_t split0 = smem_u32(&bars[2 * S + 1]);
  volatile int* ab = &abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
      mbar_init(split0 + 8 * s, 4 * 32);  // every thread of warps 2-5
    }
    mbar_init(accum, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_slot), BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        if (kb >= S && !wait_phase(empty0 + 8 * s, ((kb / S) - 1) & 1, ab)) break;
        const uint32_t st = ring + s * G::STAGE_BYTES;
        mbar_expect_tx(full0 + 8 * s, TX);
        tma_load_2d(st, &map_ahi, full0 + 8 * s, kb * BK, (int)m0);
        if (!ASPLIT) tma_load_2d(st + G::A_BYTES, &map_alo, full0 + 8 * s, kb * BK, (int)m0);
        tma_load_2d(st + 2 * G::A_BYTES, &map_b, full0 + 8 * s, kb * BK, n0);
        if (BLO) tma_load_2d(st + 2 * G::A_BYTES + G::B_BYTES, &map_blo, full0 + 8 * s, kb * BK, n0);
        issued = kb + 1;
      }
      // no copy may still be landing when the block exits: wait for the last fill of every stage
      for (int kb = issued > S ? issued - S : 0; kb < issued; ++kb) wait_drain(full0 + 8 * (kb % S), (kb / S) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, BN);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        if (!wait_phase((ASPLIT ? split0 : full0) + 8 * s, (kb / S) & 1, ab)) break;
        tc_fence_after();
        const uint32_t st = ring + s * G::STAGE_BYTES;
        const uint64_t dah = desc_sw128(st), dal = desc_sw128(st + G::A_BYTES), db = desc_sw128(st + 2 * G::A_BYTES);
        const uint64_t dbl = desc_sw128(st + 2 * G::A_BYTES + G::B_BYTES);
#pragma unroll
        for (int k = 0; k < BK / UK; ++k) {
          const uint64_t off = (uint64_t)((k * UK * 4) >> 4);  // 32-byte steps inside the swizzle span
          mma_tf32(tmem, dah + off, db + off, idesc, (kb | k) != 0 ? 1u : 0u);
          mma_tf32(tmem, dal + off, db + off, idesc, 1u);
          if (BLO) mma_tf32(tmem, dah + off, dbl + off, idesc, 1u);
        }
        mma_commit(empty0 + 8 * s);  // the stage is free once these MMAs have read it
      }
      mma_commit(accum);  // always: the read-back and the release wait on it
    }
  } else {
    if (ASPLIT) {
      // split every stage's A tile: thread t owns row t (128 bytes: eight 16-byte chunks, wherever the
      // swizzle put them, so the layout is kept); hi in place, lo into the A_lo slot
      const int t = threadIdx.x - 64;
      unsigned char* gring = dyn + (ring - smem_u32(dyn));
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        bool ok = false;
        if (lane == 0) ok = wait_phase(full0 + 8 * s, (kb / S) & 1, ab);
        if (__shfl_sync(0xffffffffu, ok ? 1 : 0, 0) == 0) break;
        float4* hi = reinterpret_cast<float4*>(gring + (size_t)s * G::STAGE_BYTES + (size_t)t * 128);
        float4* lo = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(hi) + G::A_BYTES);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = hi[c];
          const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
          hi[c] = h;
          lo[c] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
        // the tensor cores (async proxy) read what these generic stores wrote
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(split0 + 8 * s) : "memory");
      }
    }
    const int q = warp & 3;  // the tensor-memory lane quadrant this warp may read
    bool go = false;
    if (lane == 0) go = wait_phase(accum, 0, ab) && !*ab;
    go = __shfl_sync(0xffffffffu, go ? 1 : 0, 0) != 0;
    tc_fence_after();
    if (go) {
      const long long row = m0 + 32 * q + lane;
      const bool live = row < rows;
      const long long p = live ? row / plane_rows : 0;
      const long long base = p * plane_stride + (row - p * plane_rows);
      for (int c = 0; c < BN / 16; ++c) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * 16), v);
        if (live) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int j = n0 + c * 16 + i;
            if (j < ncols) {
              const float x = __uint_as_float(v[i]);
              const long long o = base + (long long)j * plane_rows;
              if (out_lo) {
                const float h = tf32_hi(x);
                out_hi[o] = h;
                out_lo[o] = x - h;
              } else {
                out_hi[o] = x;
              }
            }
          }
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if (lane == 0) wait_drain(accum, 0);  // every MMA of the block has completed
    __syncwarp();
    tmem_dealloc(tmem, BN);
  }
  if (threadIdx.x == 0 && *ab) atomicExch(err, 1);
}

// ---- host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// FP32 matrix of `nrows` rows of K values (row stride K), boxes of 32 x box_rows, 128-byte swizzle;
// rows and k beyond the matrix read as zero. A map is a pure function of (address, rows, K, box), so
// the last maps built by this host thread are kept and reused (the preconditioner calls the same few
// shapes on the same buffers at every Krylov iteration).
struct MapEntry {
  CUtensorMap map;
  const float* p;
  long long nrows;
  int K, box;
};
constexpr int kMapCache = 32;
thread_local MapEntry t_maps[kMapCache];
thread_local int t_nmaps = 0, t_next = 0;

bool make_map(CUtensorMap* m, const float* p, long long nrows, int K, int box_rows) {
  for (int i = 0; i < t_nmaps; ++i) {
    const MapEntry& e = t_maps[i];
    if (e.p == p && e.nrows == nrows && e.K == K && e.box == box_rows) {
      *m = e.map;
      return true;
    }
  }
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  if (fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  MapEntry& e = t_maps[t_next];
  t_next = (t_next + 1) % kMapCache;
  if (t_nmaps < kMapCache) ++t_nmaps;
  e.map = *m;
  e.p = p;
  e.nrows = nrows;
  e.K = K;
  e.box = box_rows;
  return true;
}

template <int BN, bool BLO, bool ASPLIT>
cudaError_t launch(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& mb, const CUtensorMap& mbl,
                   long long rows, int K, int ncols, long long plane_rows, long long plane_stride, float* out_hi,
                   float* out_lo, int* err, long long blocks, cudaStream_t st) {
  using G = Cfg<BN, BLO>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tc_axis<BN, BLO, ASPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)G::SMEM);
  });
  if (attr != cudaSuccess) return attr;
  k_tc_axis<BN, BLO, ASPLIT><<<(unsigned)blocks, THREADS, G::SMEM, st>>>(ah, al, mb, mbl, rows, K, ncols, plane_rows,
                                                                         plane_stride, out_hi, out_lo, err);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_any(bool blo, bool asplit, const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& mb,
                       const CUtensorMap& mbl, long long rows, int K, int ncols, long long plane_rows,
                       long long plane_stride, float* out_hi, float* out_lo, int* err, long long blocks,
                       cudaStream_t st) {
  if (blo)
    return asplit ? launch<BN, true, true>(ah, al, mb, mbl, rows, K, ncols, plane_rows, plane_stride, out_hi, out_lo,
                                           err, blocks, st)
                  : launch<BN, true, false>(ah, al, mb, mbl, rows, K, ncols, plane_rows, plane_stride, out_hi, out_lo,
                                            err, blocks, st);
  return asplit ? launch<BN, false, true>(ah, al, mb, mbl, rows, K, ncols, plane_rows, plane_stride, out_hi, out_lo,
                                          err, blocks, st)
                : launch<BN, false, false>(ah, al, mb, mbl, rows, K, ncols, plane_rows, plane_stride, out_hi, out_lo,
                                           err, blocks, st);
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace tc

int tc_axis_transform(const float* a_hi, const float* a_lo, long long rows, int K, const float* b, const float* b_lo,
                      int ncols, long long plane_rows, long long plane_stride, float* out_hi, float* out_lo, int* err,
                      int tile_n, cudaStream_t st) {
  using namespace tc;
  if (!a_hi || !b || !out_hi || !err || rows < 1 || K < 4 || K % 4 != 0 || ncols < 1 || plane_rows < 1 ||
      plane_stride < 0 || rows > INT_MAX - BM || ncols > INT_MAX - 256 ||
      (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256))
    return TDZ_EINVAL;
  if (!aligned16(a_hi) || (a_lo && !aligned16(a_lo)) || !aligned16(b) || (b_lo && !aligned16(b_lo)))
    return TDZ_EINVAL;
  const long long tiles_m = (rows + BM - 1) / BM;
  // default: 256-column tiles where there are enough of them to fill the device twice, else 128
  const bool wide = tile_n ? tile_n == 256 : tiles_m * ((ncols + 255) / 256) >= 2 * 148;
  const int bn = tile_n == 64 ? 64 : wide ? 256 : 128;
  const long long blocks = tiles_m * ((ncols + bn - 1) / bn);
  if (blocks > INT_MAX) return TDZ_EINVAL;
  CUtensorMap mah, mal, mb, mbl;
  if (!make_map(&mah, a_hi, rows, K, BM) || !make_map(&mal, a_lo ? a_lo : a_hi, rows, K, BM) ||
      !make_map(&mb, b, ncols, K, bn) ||
      !make_map(&mbl, b_lo ? b_lo : b, ncols, K, bn))
    return TDZ_ECUDA;
  const bool asplit = a_lo == nullptr;
  const cudaError_t e =
      bn == 64    ? launch_any<64>(b_lo != nullptr, asplit, mah, mal, mb, mbl, rows, K, ncols, plane_rows, plane_stride,
                                   out_hi, out_lo, err, blocks, st)
      : bn == 256 ? launch_any<256>(b_lo != nullptr, asplit, mah, mal, mb, mbl, rows, K, ncols, plane_rows,
                                    plane_stride, out_hi, out_lo, err, blocks, st)
                  : launch_any<128>(b_lo != nullptr, asplit, mah, mal, mb, mbl, rows, K, ncols, plane_rows,
                                    plane_stride, out_hi, out_lo, err, blocks, st);
  if (e != cudaSuccess) {
    set_error(std::string("tensor-core axis transform: ") + cudaGetErrorString(e));
    return TDZ_ECUDA;
  }
  return TDZ_OK;
}

}  // namespace tdz

// ---- C ABI (include/tdz.h)
extern "C" int tdz_tc_axis_transform(const float* a_hi, const float* a_lo, int64_t rows, int k, const float* b,
                                     const float* b_lo, int ncols, int64_t plane_rows, int64_t plane_stride,
                                     float* out_hi, float* out_lo, int tile_n, void* cuda_stream) {
  static int* d_err = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) d_err = nullptr;
    else cudaMemset(d_err, 0, sizeof(int));
  });
  if (!d_err) {
    tdz::set_error("tdz_tc_axis_transform: no device memory for the error word");
    return TDZ_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int rc = tdz::tc_axis_transform(a_hi, a_lo, rows, k, b, b_lo, ncols, plane_rows, plane_stride, out_hi, out_lo,
                                        d_err, tile_n, st);
  if (rc != TDZ_OK) return rc;
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    tdz::set_error(std::string("tdz_tc_axis_transform: ") + cudaGetErrorString(e));
    return TDZ_ECUDA;
  }
  if (herr) {
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    tdz::set_error("tdz_tc_axis_transform: a pipeline wait ran out of time");
    return TDZ_ECUDA;
  }
  return TDZ_OK;
}
