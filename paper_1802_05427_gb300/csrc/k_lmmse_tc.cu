// LS + sub-block LMMSE (Eq. 9, 12, 17) on the 5th-generation tensor cores (tcgen05).
//
// With B dividing n_sc, every (slot, user, antenna) row splits into nb blocks and all full
// blocks share W.  The LS estimates then form one matrix X with R * nb rows ("row-blocks")
// of B complex values, stored contiguously in y_pilot's layout, and the filter is the GEMM
//   H = X W^T  (complex)  =  X_r Wr^T  in the interleaved real embedding,
// X_r: rows x 2B floats (re, im, re, im, ...), Wr[2i][2j] = Re W[i][j], Wr[2i][2j+1] =
// -Im W[i][j], Wr[2i+1][2j] = Im W[i][j], Wr[2i+1][2j+1] = Re W[i][j].
//
// FP32 accuracy on TF32 tensor cores: every operand is split x = hi + lo (both TF32) and
// D = Ah Wh^T + Ah Wl^T + Al Wh^T, accumulated in FP32 in tensor memory.
//
// Persistent CTAs work through contiguous runs of tiles of 128 row-blocks (B * 1 KB,
// contiguous in memory), with three roles:
//  * a copy warp: 1-D bulk copies of raw tiles into a ring of stages, and one bulk store
//    per filtered tile, after which the stage takes the next load;
//  * 256 consumer threads, two per row-block (one per half of its reals): the LS estimate
//    y conj(p) / |p|^2, split into TF32 hi and lo in the canonical K-major layout (8-row x
//    16-byte core matrices) of one of two A buffers; then, for the previous tile, the
//    accumulator row read back from tensor memory (tcgen05.ld, TMEM lane = row-block) and
//    written over the raw stage;
//  * an MMA warp: one thread issues the MMAs of a tile (M = 128, N = 32, K = 8 each) into
//    one of two accumulators as soon as its A buffer is complete, and commits them to an
//    mbarrier.
// Only mbarriers order the roles, so the LS of tile i+1 runs while the tensor cores work
// on tile i and the copies of other tiles are in flight.

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "host_round.h"
#include "rapro_internal.h"
#include "rapro_ptx.cuh"

namespace rapro {

namespace {

constexpr int TC_ROWS = 128;        // row-blocks per tile (MMA M, TMEM lanes)
constexpr int TC_N = 32;            // MMA N: 2B <= 32 output reals, padded with zero weights
constexpr int TC_STAGES = 4;        // raw-tile ring depth
constexpr int TC_CONSUMERS = 256;    // two threads per row-block, one per half of its reals
constexpr int TC_THREADS = TC_CONSUMERS + 64;   // + one MMA warp + one copy warp

// The TF32 passes use the shared M = 128, N = 32 instruction (rapro_ptx.cuh).
static_assert(TC_ROWS == 128 && TC_N == 32, "the TF32 MMA helper is M = 128, N = 32");

// Operand forms of the filter: three TF32 passes (FP32 accuracy) or one pass of 16-bit
// operands, both A and B in the same format (BF16 or FP16), FP32 accumulation.
enum { OP_TF32X3 = 0, OP_BF16 = 1, OP_FP16 = 2 };

// Instruction descriptors: D = F32, A = B = BF16 (format 1) or FP16 (format 0), both
// K-major, M = 128, N = TC_N.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TC_N >> 3) << 17) |
                                (uint32_t(TC_ROWS >> 4) << 24);
constexpr uint32_t kIdescFp16 = (1u << 4) | (0u << 7) | (0u << 10) | (uint32_t(TC_N >> 3) << 17) |
                                (uint32_t(TC_ROWS >> 4) << 24);

template <uint32_t IDESC>
__device__ __forceinline__ void mma_f16kind(uint32_t d_tmem, uint64_t a, uint64_t b, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate ? 1 : 0)
      : "memory");
}

// Two floats rounded to nearest even into one 32-bit word, the first at the lower address.
template <int OP>
__device__ __forceinline__ uint32_t pack16x2(float lo, float hi) {
  if constexpr (OP == OP_FP16) return pack_f16x2(lo, hi);
  else return pack_bf16x2(lo, hi);
}

}  // namespace

// KR: reals per row-block, 2B padded to the MMA's K step (8 for TF32, 16 for 16-bit).
// OP: the operand form; OP_BF16 / OP_FP16 is one 16-bit pass (the precision form) instead
// of the three TF32 passes.
template <int KR, int OP>
__global__ void __launch_bounds__(TC_THREADS, 1) lmmse_tc_kernel(const float2* __restrict__ y,
                                                              const float2* __restrict__ pil,
                                                              float2* __restrict__ out, int M, int N, int B,
                                                              long long n_rb, int n_tiles, int* status,
                                                              const void* __restrict__ w_tc) {
  constexpr bool BF = OP != OP_TF32X3;                          // one 16-bit pass
  static_assert(KR % (BF ? 16 : 8) == 0 && KR <= 32, "2B padded to the K step, at most 32");
  constexpr int ELT = BF ? 2 : 4;                               // operand bytes
  constexpr int CE = 16 / ELT;                                  // operand elements per 16-byte core row
  constexpr uint32_t SBO = (KR / CE) * 128;                     // 8-row group stride (A and B)
  constexpr int A_BYTES = TC_ROWS * KR * ELT;
  constexpr int B_BYTES = TC_N * KR * ELT;
  constexpr int NA = BF ? 1 : 2;                                // A parts: BF16, or TF32 hi and lo
  constexpr int KSTEPS = KR / (2 * CE);                         // MMAs of K = 2 core columns (32 bytes)
  constexpr int KQ = KR / 4;                                    // float4 (2 complex) per row-block
  constexpr int KH = KQ / 2;                                    // float4 per consumer thread
  static_assert(!BF || KH % 2 == 0, "a BF16 core row holds two float4 of reals");
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);           // [TC_STAGES] raw tile landed
  uint64_t* epi = full + TC_STAGES;                             // [TC_STAGES] tile written back
  uint64_t* aready = epi + TC_STAGES;                           // [2] A buffer holds a tile
  uint64_t* done = aready + 2;                                  // [2] MMAs of an A buffer finished
  uint64_t* wbar = done + 2;                                    // weights landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  unsigned char* sA = smem + 1024;                              // [2 buffers][NA parts][A_BYTES]
  unsigned char* sBh = sA + 2 * NA * A_BYTES;                   // weights (TF32: hi, then lo)
  float2* raw = reinterpret_cast<float2*>(sBh + NA * B_BYTES);  // [TC_STAGES][TC_ROWS * B]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile_elems = TC_ROWS * B;
  const int nb = N / B;

  if (tid == 0) {
    for (int st = 0; st < TC_STAGES; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&epi[st], TC_CONSUMERS);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&aready[b], TC_CONSUMERS);
      mbar_init(&done[b], 1);
    }
    mbar_init(wbar, 1);
    *s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {   // two accumulators of TC_N columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // Each CTA takes a contiguous run of tiles: its row-blocks then share few pilot rows,
  // which stay in L1 after the first tile.
  const int t_begin = int((long long)n_tiles * blockIdx.x / gridDim.x);
  const int my_tiles = int((long long)n_tiles * (blockIdx.x + 1) / gridDim.x) - t_begin;
  auto tile_of = [&](int it) { return t_begin + it; };
  auto tile_count = [&](int it) -> int {
    const long long left = n_rb - (long long)tile_of(it) * TC_ROWS;
    return int(left < TC_ROWS ? left : TC_ROWS);
  };
  auto give_up = [&]() {
    *s_abort = 1;
    atomicExch(status, int(RAPRO_ERR_TIMEOUT));
  };

  if (warp == TC_CONSUMERS / 32 + 1) {
    // ------------------------------------------------ copy warp: loads and stores
    if (lane == 0 && my_tiles > 0) {
      auto issue = [&](int it) {
        const int st = it % TC_STAGES;
        const uint32_t bytes = uint32_t(tile_count(it)) * B * sizeof(float2);
        mbar_arrive_expect_tx(&full[st], bytes);
        bulk_load(raw + size_t(st) * tile_elems, y + (size_t)tile_of(it) * tile_elems, bytes, &full[st]);
      };
      // The weights arrive already in the canonical layout (NA * B_BYTES).
      mbar_arrive_expect_tx(wbar, NA * B_BYTES);
      bulk_load(sBh, w_tc, NA * B_BYTES, wbar);
      int issued = 0;
      for (; issued < TC_STAGES && issued < my_tiles; ++issued) issue(issued);
      bool bad = false;
      for (int it = 0; it < my_tiles; ++it) {
        const int st = it % TC_STAGES;
        if (!mbar_wait_bounded(&epi[st], uint32_t(it / TC_STAGES) & 1u) || *s_abort) {
          bad = true;
          break;
        }
        bulk_store(out + (size_t)tile_of(it) * tile_elems, raw + size_t(st) * tile_elems,
                   uint32_t(tile_count(it)) * B * sizeof(float2));
        bulk_commit();
        if (it + TC_STAGES < my_tiles) {
          bulk_wait_read<0>();                 // the store has read the stage
          issue(issued);
          ++issued;
        }
      }
      bulk_wait_all();
      // Let every load land before the CTA exits (on the normal path all have been consumed):
      // load j of stage s is phase j of full[s], the last one (issued - 1 - s) / TC_STAGES.
      for (int s2 = 0; s2 < TC_STAGES && s2 < issued; ++s2)
        (void)mbar_wait_bounded(&full[s2], uint32_t((issued - 1 - s2) / TC_STAGES) & 1u);
      (void)mbar_wait_bounded(wbar, 0u);
      if (bad) give_up();
    }
  } else if (warp == TC_CONSUMERS / 32) {
    // ------------------------------------------------ MMA warp: one thread issues
    if (lane == 0 && my_tiles > 0) {
      bool bad = !mbar_wait_bounded(wbar, 0u);
      int issued = 0;
      for (int it = 0; it < my_tiles && !bad; ++it) {
        const int buf = it & 1;
        if (!mbar_wait_bounded(&aready[buf], uint32_t(it >> 1) & 1u) || *s_abort) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // TF32: D[buf] = Ah Wh^T + Ah Wl^T + Al Wh^T;  BF16: D[buf] = A W^T.  K = KR in
        // steps of two core columns.
        const unsigned char* ah = sA + buf * NA * A_BYTES;
        const unsigned char* al = ah + A_BYTES;
        const uint32_t d = tmem + uint32_t(buf * TC_N);
#pragma unroll
        for (int kg = 0; kg < KSTEPS; ++kg) {
          const uint64_t dah = smem_desc_kmajor(ah + kg * 256, 128, SBO), dbh = smem_desc_kmajor(sBh + kg * 256, 128, SBO);
          if (BF) {
            mma_f16kind<OP == OP_FP16 ? kIdescFp16 : kIdescBf16>(d, dah, dbh, kg > 0);
          } else {
            const uint64_t dal = smem_desc_kmajor(al + kg * 256, 128, SBO);
            const uint64_t dbl = smem_desc_kmajor(sBh + B_BYTES + kg * 256, 128, SBO);
            mma_tf32_m128n32(d, dah, dbh, kg > 0);
            mma_tf32_m128n32(d, dah, dbl, true);
            mma_tf32_m128n32(d, dal, dbh, true);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done[buf]))
                     : "memory");
        ++issued;
      }
      if (bad) {
        // The tensor cores finish in order: wait for the last group before TMEM is freed.
        if (issued > 0) (void)mbar_wait_bounded(&done[(issued - 1) & 1], uint32_t((issued - 1) >> 1) & 1u);
        give_up();
      }
    }
  } else {
    // ------------------------------------------------ consumers: LS + split, read-back
    const int r = tid & (TC_ROWS - 1), half = tid / TC_ROWS;   // row-block of the tile, half of it
    // This thread's row-block of tile it: rb = row * nb + b, row = tk * M + m (tk = slot-user).
    // Tiles of a CTA are consecutive, so rb advances by TC_ROWS per tile and the quotients are
    // carried along instead of divided again (a division only when m passes M).
    uint32_t p_b = 0, p_tk = 0, p_m = 0;
    const uint32_t q_rows = uint32_t(TC_ROWS) / uint32_t(nb), r_rows = uint32_t(TC_ROWS) % uint32_t(nb);
    {
      const uint32_t rb0 = uint32_t(tile_of(0)) * TC_ROWS + uint32_t(r);   // n_rb < 2^31
      const uint32_t row0 = rb0 / uint32_t(nb);
      p_b = rb0 - row0 * uint32_t(nb);
      p_tk = row0 / uint32_t(M);
      p_m = row0 - p_tk * uint32_t(M);
    }
    auto advance_row_block = [&]() {
      p_b += r_rows;
      uint32_t dr = q_rows;
      if (p_b >= uint32_t(nb)) {
        p_b -= uint32_t(nb);
        ++dr;
      }
      p_m += dr;
      if (p_m >= uint32_t(M)) {
        p_tk += p_m / uint32_t(M);
        p_m %= uint32_t(M);
      }
    };
    // Pilots of this thread's row-block of tile it (B complex, two per float4); called for
    // it = 0, 1, 2, ... in order, each call after the first moving on by one tile.
    auto load_pilots = [&](int it, float4 (&pv)[KH]) {
      if (it > 0) advance_row_block();
      if (it >= my_tiles || r >= tile_count(it)) return;
      const float4* pr = reinterpret_cast<const float4*>(pil + size_t(p_tk) * N + size_t(p_b) * B);
#pragma unroll
      for (int j = 0; j < KH; ++j) {
        const int kg = half * KH + j;
        if (2 * kg < B) pv[j] = __ldg(pr + kg);
      }
    };
    // LS estimate (y conj(p) / |p|^2) split into TF32 hi and lo, canonical K-major layout.
    auto ls_split = [&](int it, const float4 (&pv)[KH], int buf) {
      unsigned char* ah = sA + buf * NA * A_BYTES;
      unsigned char* al = ah + A_BYTES;
      const bool live = r < tile_count(it);
      const float4* x4 = reinterpret_cast<const float4*>(raw + size_t(it % TC_STAGES) * tile_elems + r * B);
      float4 q[KH];
#pragma unroll
      for (int j = 0; j < KH; ++j) {
        const int kg = half * KH + j;
        q[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live && 2 * kg < B) {
          const float4 x = x4[kg], p = pv[j];
          const float i0 = __fdividef(1.0f, fmaf(p.x, p.x, p.y * p.y));
          const float i1 = __fdividef(1.0f, fmaf(p.z, p.z, p.w * p.w));
          q[j] = make_float4(fmaf(x.x, p.x, x.y * p.y) * i0, fmaf(x.y, p.x, -x.x * p.y) * i0,
                             fmaf(x.z, p.z, x.w * p.w) * i1, fmaf(x.w, p.z, -x.z * p.w) * i1);
        }
      }
      if (BF) {
        // Four complex (8 BF16) per 16-byte core row.
#pragma unroll
        for (int j = 0; j < KH; j += 2) {
          const int c = (half * KH + j) / 2;
          const uint4 v = make_uint4(pack16x2<OP>(q[j].x, q[j].y), pack16x2<OP>(q[j].z, q[j].w),
                                     pack16x2<OP>(q[j + 1].x, q[j + 1].y), pack16x2<OP>(q[j + 1].z, q[j + 1].w));
          *reinterpret_cast<uint4*>(ah + (r / 8) * SBO + c * 128 + (r % 8) * 16) = v;
        }
      } else {
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int kg = half * KH + j;
          const float4 h = make_float4(tf32_trunc(q[j].x), tf32_trunc(q[j].y), tf32_trunc(q[j].z), tf32_trunc(q[j].w));
          const float4 l = make_float4(q[j].x - h.x, q[j].y - h.y, q[j].z - h.z, q[j].w - h.w);
          const int off = (r / 8) * SBO + kg * 128 + (r % 8) * 16;
          *reinterpret_cast<float4*>(ah + off) = h;
          *reinterpret_cast<float4*>(al + off) = l;
        }
      }
    };
    // Accumulator row r (this warp's quarter of the TMEM lanes) over the raw tile; the
    // branch on half is warp-uniform and keeps every register index static.
    auto epilogue = [&](int it) -> bool {
      const int buf = it & 1;
      if (!mbar_wait_bounded(&done[buf], uint32_t(it >> 1) & 1u)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t v[32];
      tmem_ld32(tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(buf * TC_N), v);
      float4* o4 = reinterpret_cast<float4*>(raw + size_t(it % TC_STAGES) * tile_elems + r * B);
      const bool live = r < tile_count(it);
      auto put = [&](auto hc) {
        constexpr int H = decltype(hc)::value;
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int kg = H * KH + j;
          if (live && 2 * kg < B)
            o4[kg] = make_float4(__uint_as_float(v[4 * kg]), __uint_as_float(v[4 * kg + 1]),
                                 __uint_as_float(v[4 * kg + 2]), __uint_as_float(v[4 * kg + 3]));
        }
      };
      if (half == 0) put(std::integral_constant<int, 0>{});
      else put(std::integral_constant<int, 1>{});
      fence_proxy_async_shared();              // the bulk store reads what was written here
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&epi[it % TC_STAGES]);
      return true;
    };
    float4 pv[KH];
#pragma unroll
    for (int j = 0; j < KH; ++j) pv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    load_pilots(0, pv);
    bool bad = false;
    // Tile it's LS runs while the tensor cores work on tile it - 1.
    for (int it = 0; it < my_tiles; ++it) {
      if (*s_abort || !mbar_wait_bounded(&full[it % TC_STAGES], uint32_t(it / TC_STAGES) & 1u)) {
        bad = true;
        break;
      }
      ls_split(it, pv, it & 1);               // A buffer it & 1 was last read by MMA it - 2
      load_pilots(it + 1, pv);
      fence_proxy_async_shared();              // the MMAs read what was written here
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&aready[it & 1]);
      if (it >= 1 && !epilogue(it - 1)) {
        bad = true;
        break;
      }
    }
    if (!bad && my_tiles > 0 && !epilogue(my_tiles - 1)) bad = true;
    if (bad) give_up();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N) : "memory");
}

template <int KR, int OP>
static size_t tc_smem_bytes(int B) {
  const size_t elt = OP != OP_TF32X3 ? 2 : 4, na = OP != OP_TF32X3 ? 1 : 2;
  return 1024 + 2 * na * size_t(TC_ROWS) * KR * elt + na * size_t(TC_N) * KR * elt +
         size_t(TC_STAGES) * TC_ROWS * B * sizeof(float2);
}


// Reals per row-block: 2B padded to the K step (8 for TF32, 16 for BF16).
static int kr_for(int B, bool half) { return half ? (2 * B + 15) / 16 * 16 : (2 * B + 7) / 8 * 8; }

template <int KR, int OP>
static cudaError_t launch_tc(const Plan& pl, const float2* y, const float2* pil, float2* out, cudaStream_t st) {
  const int B = pl.B, M = pl.p.M, N = pl.p.n_sc, R = pl.T * pl.p.K * pl.p.M;
  const long long n_rb = (long long)R * (N / B);
  const int n_tiles = int((n_rb + TC_ROWS - 1) / TC_ROWS);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  // SM count, shared memory per SM, reserved shared memory and this kernel's registers, read
  // once per device (the first launch may not be inside a stream capture).
  struct Attrs { int sms = 148, smem_sm = 0, reserved = 0, regs = 1; };
  static Attrs attrs[64];
  static std::once_flag once[64];
  std::call_once(once[dev], [dev] {
    Attrs& a = attrs[dev];
    cudaDeviceGetAttribute(&a.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&a.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&a.reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, lmmse_tc_kernel<KR, OP>) == cudaSuccess) a.regs = std::max(fa.numRegs, 1);
  });
  const Attrs& at = attrs[dev];
  const int sms = at.sms;
  const size_t smem = tc_smem_bytes<KR, OP>(B);
  // Resident CTAs per SM: shared memory, threads (2048 per SM), registers (64 K, allocated
  // per warp in units of 8 per thread) and tensor memory (512 columns).
  const int regs_warp = ((at.regs + 7) / 8 * 8) * 32;
  int per_sm = int(size_t(at.smem_sm) / (smem + size_t(at.reserved)));
  per_sm = std::max(1, std::min({per_sm, 2048 / TC_THREADS, 512 / (2 * TC_N), 65536 / (regs_warp * (TC_THREADS / 32))}));
  if (pl.est_ctas_per_sm > 0) per_sm = std::min(per_sm, pl.est_ctas_per_sm);
  const int grid = std::min(n_tiles, per_sm * sms);
  lmmse_tc_kernel<KR, OP><<<grid, TC_THREADS, smem, st>>>(y, pil, out, M, N, B, n_rb, n_tiles, pl.d_status,
                                                            pl.d_w_tc);
  return cudaGetLastError();
}

bool lmmse_tc_shape_ok(const Plan& pl) {
  if (pl.B < 2) return false;
  const long long n_rb = (long long)pl.T * pl.p.K * pl.p.M * (pl.p.n_sc / pl.B);
  return pl.B % 2 == 0 && pl.B <= 16 && pl.tail == 0 && n_rb < (1ll << 31);
}

// The filter as the MMA's B operand: Wr (TC_N x KR reals, zero padded) in the canonical
// K-major layout: TF32 hi part followed by its lo part, or one BF16 / FP16 part (raw bytes).
void build_lmmse_tc_weights(const Plan& pl, std::vector<unsigned char>& out) {
  const bool bf = half_precision(pl.p), f16 = pl.p.precision == RAPRO_PREC_FP16;
  const int B = pl.B, KR = kr_for(B, bf), elt = bf ? 2 : 4, ce = 16 / elt;
  const int SBO = (KR / ce) * 128, part = TC_N * KR * elt;
  out.assign(size_t(bf ? 1 : 2) * part, 0);
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) {
      const float2 v = pl.w_main[size_t(i) * B + j];
      const float vals[2][2] = {{v.x, -v.y}, {v.y, v.x}};   // [out re/im][in re/im]
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
          const int n = 2 * i + a, k = 2 * j + c;
          const size_t off = size_t((n / 8) * SBO + (k / ce) * 128 + (n % 8) * 16 + (k % ce) * elt);
          const float f = vals[a][c];
          if (bf) {
            const uint16_t h = f16 ? f16_round_host(f) : bf16_round_host(f);
            std::memcpy(&out[off], &h, 2);
          } else {
            const float h = tf32_round_host(f), l = tf32_round_host(f - h);
            std::memcpy(&out[off], &h, 4);
            std::memcpy(&out[part + off], &l, 4);
          }
        }
    }
}

bool lmmse_tc_ok(const Plan& pl, const float2* y, const float2* pil, const float2* out) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(pil) |
                      reinterpret_cast<uintptr_t>(out);
  return pil != nullptr && pl.d_w_tc != nullptr && (a & 15) == 0 && lmmse_tc_shape_ok(pl);
}

cudaError_t launch_lmmse_tc(const Plan& pl, const float2* y, const float2* pil, float2* out, cudaStream_t st) {
  if (pl.p.precision == RAPRO_PREC_BF16)
    return kr_for(pl.B, true) == 16 ? launch_tc<16, OP_BF16>(pl, y, pil, out, st)
                                    : launch_tc<32, OP_BF16>(pl, y, pil, out, st);
  if (pl.p.precision == RAPRO_PREC_FP16)
    return kr_for(pl.B, true) == 16 ? launch_tc<16, OP_FP16>(pl, y, pil, out, st)
                                    : launch_tc<32, OP_FP16>(pl, y, pil, out, st);
  switch (kr_for(pl.B, false)) {
    case 8: return launch_tc<8, OP_TF32X3>(pl, y, pil, out, st);
    case 16: return launch_tc<16, OP_TF32X3>(pl, y, pil, out, st);
    case 24: return launch_tc<24, OP_TF32X3>(pl, y, pil, out, st);
    default: return launch_tc<32, OP_TF32X3>(pl, y, pil, out, st);
  }
}

cudaError_t prepare_lmmse_tc(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(lmmse_tc_kernel<8, OP_TF32X3>, A, int(tc_smem_bytes<8, OP_TF32X3>(4)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lmmse_tc_kernel<16, OP_TF32X3>, A, int(tc_smem_bytes<16, OP_TF32X3>(8)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lmmse_tc_kernel<24, OP_TF32X3>, A, int(tc_smem_bytes<24, OP_TF32X3>(12)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lmmse_tc_kernel<32, OP_TF32X3>, A, int(tc_smem_bytes<32, OP_TF32X3>(16)));
    for (int op : {int(OP_BF16), int(OP_FP16)}) {
      if (e != cudaSuccess) break;
      e = op == OP_BF16 ? cudaFuncSetAttribute(lmmse_tc_kernel<16, OP_BF16>, A, int(tc_smem_bytes<16, OP_BF16>(8)))
                        : cudaFuncSetAttribute(lmmse_tc_kernel<16, OP_FP16>, A, int(tc_smem_bytes<16, OP_FP16>(8)));
      if (e == cudaSuccess)
        e = op == OP_BF16 ? cudaFuncSetAttribute(lmmse_tc_kernel<32, OP_BF16>, A, int(tc_smem_bytes<32, OP_BF16>(16)))
                          : cudaFuncSetAttribute(lmmse_tc_kernel<32, OP_FP16>, A, int(tc_smem_bytes<32, OP_FP16>(16)));
    }
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
