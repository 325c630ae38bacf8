// LS + sub-block LMMSE (Eq. 9, 12, 17) for large blocks as a GEMM on the 5th-generation
// tensor cores (tcgen05): FP32 accuracy from three TF32 passes, or the precision forms'
// single pass of BF16 / FP16 operands.
//
// With B dividing n_sc all blocks share W, and block b of every row r = (slot, user,
// antenna) is one row of the product
//   H_b = X_b W^T (complex)  =  X_r,b Wr^T  in the interleaved real embedding,
// K = 2B input reals, N = 2B output reals (Wr as in k_lmmse_tc.cu).  For B > 16 the whole
// W no longer fits beside the operands, so an output tile is 128 rows x NT output reals of
// one block, computed over K in chunks of 32 reals (16 subcarriers); persistent CTAs take
// runs of tiles:
//  * a copy warp brings each raw chunk (128 rows x 16 complex of y_pilot, or of h_ls) by a
//    2-D TMA box into a 4-stage ring, and the matching chunk of Wr (NT x 32 reals, TF32 hi
//    then lo or one 16-bit part, laid out on the host in the canonical K-major layout) by
//    one bulk copy into one of two W buffers (a single column tile's W stays resident);
//  * 256 consumer threads apply LS (y conj(p) / |p|^2) and split each value into TF32
//    hi + lo (both rounded to nearest), or round it to BF16 / FP16, in the canonical layout
//    of one of two A buffers;
//  * one MMA thread issues the chunk's K-steps (TF32: 4 x 3 passes Ah Wh + Ah Wl + Al Wh,
//    K = 8; 16-bit: 2 x 1 pass, K = 16; M = 128, N = NT) into one of two FP32 accumulators in
//    tensor memory and commits each chunk to an mbarrier, which frees that chunk's A and W
//    buffers;
// and every G_DR chunks the consumers drain the accumulator (TMEM lane = row) into FP32
// registers while the next group's MMAs run in the other one, storing their row's outputs
// after a tile's last group.  Only mbarriers order the roles; every wait is bounded.
// That kernel serves the TF32 form.  The 16-bit forms round each LS value once, in a staging
// pass that writes the A chunks of every row tile in the canonical layout to the plan's
// buffer (tcg_stage_kernel), and lmmse_tcg16_kernel then feeds A and W chunks to tcgen05
// by bulk copies alone, with 256-column output tiles from B = 128 and one drain per tile.

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "host_round.h"
#include "rapro_internal.h"
#include "rapro_ptx.cuh"

namespace rapro {

namespace {

constexpr int G_ROWS = 128;                     // rows per tile (MMA M, TMEM lanes)
constexpr int G_KC = 32;                        // input reals per K chunk (16 subcarriers)
constexpr int G_STAGES = 4;                     // raw-chunk ring depth
constexpr int G_CONSUMERS = 256;
constexpr int G_THREADS = G_CONSUMERS + 64;     // + one MMA warp + one copy warp
// Operand forms: three TF32 passes (FP32 accuracy) or one pass of BF16 / FP16 operands.
enum { G_TF32X3 = 0, G_BF16 = 1, G_FP16 = 2 };
__host__ __device__ constexpr int g_elt(int op) { return op == G_TF32X3 ? 4 : 2; }
// 8-row group stride of both operands (a chunk row is 32 reals = 32 * elt bytes)
__host__ __device__ constexpr uint32_t g_sbo(int op) { return uint32_t(G_KC * g_elt(op) / 16) * 128; }
__host__ __device__ constexpr int g_parts(int op) { return op == G_TF32X3 ? 2 : 1; }   // hi, lo / one
__host__ __device__ constexpr int g_a_part(int op) { return G_ROWS * G_KC * g_elt(op); }
constexpr int G_RAW = G_ROWS * (G_KC / 2) * 8;  // one raw chunk (bytes)
// The tensor cores' FP32 accumulation of one sum loses accuracy linearly in its length, so
// in the TF32 form (FP32 accuracy) every G_DR chunks (K = 128 reals) the accumulator is
// drained into FP32 registers (rounded to nearest) and the next group starts afresh in the
// other accumulator.  The 16-bit forms (operands rounded to 2^-9 / 2^-11; lmmse_tcg16_kernel)
// accumulate a tile's whole K in one accumulator and drain it once.
constexpr int G_DR = 4;

template <int NT, int OP>
__host__ __device__ constexpr uint32_t idesc_g() {
  // D = F32; A = B = TF32 (format 2 of kind::tf32) or BF16 (1) / FP16 (0) of kind::f16;
  // both K-major, M = 128, N = NT.
  return (1u << 4) | (uint32_t(OP == G_TF32X3 ? 2 : OP == G_BF16 ? 1 : 0) << 7) |
         (uint32_t(OP == G_TF32X3 ? 2 : OP == G_BF16 ? 1 : 0) << 10) | (uint32_t(NT >> 3) << 17) |
         (uint32_t(G_ROWS >> 4) << 24);
}

// One K step (8 TF32 or 16 BF16 / FP16 values, 32 bytes of each row).
template <int NT, int OP>
__device__ __forceinline__ void mma_g(uint32_t d_tmem, uint64_t a, uint64_t b, bool accumulate) {
  if constexpr (OP == G_TF32X3)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_g<NT, OP>()), "r"(accumulate ? 1 : 0)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_g<NT, OP>()), "r"(accumulate ? 1 : 0)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// x rounded to nearest at TF32 (ties away from zero): rounded hi and lo parts leave unbiased
// residuals of at most 2^-22 |x| (a truncating split biases them; the tensor cores' own
// accumulation error over a long K is bounded by draining, G_DR).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__host__ __device__ constexpr int tmem_cols(int nt) { return nt <= 32 ? 32 : nt <= 64 ? 64 : nt <= 128 ? 128 : 256; }

}  // namespace

// NT: output reals per tile (a multiple of 32, at most 128).  LS: the input is y_pilot and
// LS is applied on load (else the input is h_ls).  OP: operand form (G_TF32X3, G_BF16,
// G_FP16; the 16-bit forms are one pass with no lo parts).  Persistent: CTA i takes the
// contiguous run of output tiles [n_tiles i / grid, n_tiles (i + 1) / grid), tile index =
// (block, row tile, column tile) with the column tile fastest (the row tile's chunks stay in L2 for the
// next column tile); the chunks of all its tiles form one stream through the ring, and two
// accumulators in tensor memory let one drain group's read-back overlap the next group's
// MMAs.
template <int NT, bool LS, int OP>
__global__ void __launch_bounds__(G_THREADS, 1)
    lmmse_tcg_kernel(const __grid_constant__ CUtensorMap map_x, const float2* __restrict__ pil,
                     float2* __restrict__ out, const unsigned char* __restrict__ w_tiles, int R, int M, int N,
                     int B, int n_kc, int n_rt, int n_ct, int n_tiles, int w_resident, int* status) {
  static_assert(NT % 32 == 0 && NT <= 128, "NT: 32-column read-back groups");
  constexpr int ELT = g_elt(OP), NP = g_parts(OP), G_A_PART = g_a_part(OP);
  constexpr uint32_t G_SBO = g_sbo(OP);
  constexpr int W_PART = NT * G_KC * ELT;          // one part of a W chunk (bytes)
  constexpr int KSTEPS = G_KC * ELT / 32;          // MMAs per chunk and pass (32 bytes of K each)
  constexpr int TCOLS = 2 * tmem_cols(NT);         // two accumulators
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);   // [G_STAGES] raw chunk landed
  uint64_t* rawfree = full + G_STAGES;                  // [G_STAGES] consumers done with it
  uint64_t* aready = rawfree + G_STAGES;                // [2] A buffer holds a chunk
  uint64_t* wfull = aready + 2;                         // [2] W buffer landed
  uint64_t* done = wfull + 2;                           // [2] MMAs of a chunk finished
  uint64_t* drained = done + 2;                         // [2] accumulator read back
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 2);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // W: two buffers streaming the column tile's chunks, or (w_resident: one column tile whose
  // n_kc chunks all fit) every chunk loaded once for the whole run.
  unsigned char* sA = smem + 1024;                      // [2][NP][G_A_PART]
  unsigned char* sW = sA + 2 * NP * G_A_PART;           // [2 or n_kc][NP][W_PART]
  unsigned char* sRaw = sW + (w_resident ? n_kc : 2) * NP * W_PART;   // [G_STAGES][G_RAW]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t_begin = int((long long)n_tiles * blockIdx.x / gridDim.x);
  const int my_tiles = int((long long)n_tiles * (blockIdx.x + 1) / gridDim.x) - t_begin;
  const int n_q = my_tiles * n_kc;                      // chunks of the CTA's stream
  // tile li of this CTA -> (block, first row, column tile)
  auto tile = [&](int li, int& b, int& r0, int& ct) {
    const int t = t_begin + li;
    ct = t % n_ct;
    const int rest = t / n_ct;
    r0 = (rest % n_rt) * G_ROWS;
    b = rest / n_rt;
  };

  if (tid == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&rawfree[s], G_CONSUMERS);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&aready[i], G_CONSUMERS);
      mbar_init(&wfull[i], 1);
      mbar_init(&done[i], 1);
      mbar_init(&drained[i], G_CONSUMERS);
    }
    *s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(uint32_t(TCOLS))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&]() {
    *s_abort = 1;
    atomicExch(status, int(RAPRO_ERR_TIMEOUT));
  };

  if (warp == G_CONSUMERS / 32 + 1) {
    // ------------------------------------------------ copy warp: raw chunks and W chunks
    if (lane == 0 && n_q > 0) {
      prefetch_tensormap(&map_x);
      int raw_issued = 0, w_issued = 0;
      bool bad = false;
      if (w_resident) {                          // column tile 0: all its chunks, once
        mbar_arrive_expect_tx(&wfull[0], uint32_t(n_kc) * NP * W_PART);
        bulk_load(sW, w_tiles, uint32_t(n_kc) * NP * W_PART, &wfull[0]);
        w_issued = 1;
      }
      for (int q = 0; q < n_q && !bad; ++q) {
        const int li = q / n_kc, c = q - li * n_kc, s = q % G_STAGES, wb = q & 1;
        int b, r0, ct;
        tile(li, b, r0, ct);
        if (q >= G_STAGES && !mbar_wait_bounded(&rawfree[s], uint32_t(q / G_STAGES - 1) & 1u)) bad = true;
        if (!bad) {
          mbar_arrive_expect_tx(&full[s], G_RAW);
          tma_load_2d(sRaw + s * G_RAW, &map_x, &full[s], b * B + c * (G_KC / 2), r0);
          ++raw_issued;
        }
        // W buffer wb was last read by the MMAs of chunk q - 2
        if (!w_resident) {
          if (!bad && q >= 2 && !mbar_wait_bounded(&done[wb], uint32_t((q - 2) >> 1) & 1u)) bad = true;
          if (!bad) {
            mbar_arrive_expect_tx(&wfull[wb], NP * W_PART);
            bulk_load(sW + wb * NP * W_PART, w_tiles + (size_t(ct) * n_kc + c) * NP * W_PART, NP * W_PART,
                      &wfull[wb]);
            ++w_issued;
          }
        }
        if (*s_abort) bad = true;
      }
      // Let the copies in flight land before the CTA moves on (all consumed on the normal path).
      for (int s = 0; s < G_STAGES && s < raw_issued; ++s)
        (void)mbar_wait_bounded(&full[s], uint32_t((raw_issued - 1 - s) / G_STAGES) & 1u);
      for (int i = 0; i < 2 && i < w_issued; ++i)
        (void)mbar_wait_bounded(&wfull[i], uint32_t((w_issued - 1 - i) >> 1) & 1u);
      if (bad) give_up();
    }
  } else if (warp == G_CONSUMERS / 32) {
    // ------------------------------------------------ MMA warp: one thread issues
    if (lane == 0 && n_q > 0) {
      int issued = 0;
      bool bad = false;
      const int gpt = (n_kc + G_DR - 1) / G_DR;         // drain groups per tile
      for (int q = 0; q < n_q; ++q) {
        const int li = q / n_kc, c = q - li * n_kc, ab = q & 1;
        const int gg = li * gpt + c / G_DR;             // group of the CTA's stream
        // accumulator gg & 1 was last drained for group gg - 2
        if (c % G_DR == 0 && gg >= 2 && !mbar_wait_bounded(&drained[gg & 1], uint32_t((gg - 2) >> 1) & 1u)) {
          bad = true;
          break;
        }
        const bool w_ok = w_resident ? (q > 0 || mbar_wait_bounded(&wfull[0], 0u))
                                     : mbar_wait_bounded(&wfull[ab], uint32_t(q >> 1) & 1u);
        if (!mbar_wait_bounded(&aready[ab], uint32_t(q >> 1) & 1u) || !w_ok || *s_abort) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char* ah = sA + ab * NP * G_A_PART;
        const unsigned char* al = ah + G_A_PART;         // TF32 only
        const unsigned char* wh = sW + (w_resident ? c : ab) * NP * W_PART;
        const unsigned char* wl = wh + W_PART;           // TF32 only
        const uint32_t d = tmem + uint32_t((gg & 1) * tmem_cols(NT));
#pragma unroll
        for (int ks = 0; ks < KSTEPS; ++ks) {
          const uint64_t dah = smem_desc_kmajor(ah + ks * 256, 128, G_SBO);
          const uint64_t dwh = smem_desc_kmajor(wh + ks * 256, 128, G_SBO);
          mma_g<NT, OP>(d, dah, dwh, c % G_DR > 0 || ks > 0);
          if constexpr (OP == G_TF32X3) {
            mma_g<NT, OP>(d, dah, smem_desc_kmajor(wl + ks * 256, 128, G_SBO), true);
            mma_g<NT, OP>(d, smem_desc_kmajor(al + ks * 256, 128, G_SBO), dwh, true);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done[ab]))
                     : "memory");
        ++issued;
      }
      // The tensor cores finish in order: the last group done means TMEM may be freed.
      if (issued > 0) (void)mbar_wait_bounded(&done[(issued - 1) & 1], uint32_t((issued - 1) >> 1) & 1u);
      if (bad) give_up();
    }
  } else {
    // ------------------------------------------------ consumers: LS + split, read-back
    bool bad = false;
    // Drain of group gg (tile gg / gpt): warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows) and
    // 32-column groups w / 4 and w / 4 + 2 of accumulator gg & 1 and adds them to its
    // registers; after a tile's last group the registers (16 complex outputs of the row per
    // column group) are stored and cleared.  Waits for the MMAs of the group's last chunk,
    // then frees the accumulator.
    const int gpt = (n_kc + G_DR - 1) / G_DR;
    float acc_r[2][32];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 32; ++j) acc_r[i][j] = 0.f;
    auto drain = [&](int gg) -> bool {
      const int li = gg / gpt, gc = gg - li * gpt;
      const int ql = li * n_kc + min((gc + 1) * G_DR, n_kc) - 1;
      if (!mbar_wait_bounded(&done[ql & 1], uint32_t(ql >> 1) & 1u)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int rq = warp & 3;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int g = (warp >> 2) + 2 * i;
        if (g < NT / 32) {
          uint32_t v[32];
          tmem_ld32(tmem + (uint32_t(32 * rq) << 16) + uint32_t((gg & 1) * tmem_cols(NT) + 32 * g), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) acc_r[i][j] += __uint_as_float(v[j]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&drained[gg & 1]);
      if (gc == gpt - 1) {
        int b, r0, ct;
        tile(li, b, r0, ct);
        const int row = r0 + 32 * rq + lane;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int g = (warp >> 2) + 2 * i;
          const int j0 = (ct * NT + 32 * g) >> 1;     // first complex output of the group
          if (g < NT / 32 && row < R) {
            // pairs of outputs as 16-byte stores (row * N + b * B + j0 is even; so is B)
            float4* o = reinterpret_cast<float4*>(out + size_t(row) * N + size_t(b) * B + j0);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j0 + 2 * j < B) o[j] = make_float4(acc_r[i][4 * j], acc_r[i][4 * j + 1], acc_r[i][4 * j + 2], acc_r[i][4 * j + 3]);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) acc_r[i][j] = 0.f;
        }
      }
      return true;
    };
    // Element map of a chunk (128 rows x 8 float4 of two subcarriers): warp w, lane l takes
    // rows (2w + u) * 8 + (l & 7) and float4 columns c4 = ((l >> 3) + 4h + row) & 7 (u, h in
    // {0, 1}), so both the raw reads (row stride 128 bytes) and the canonical A writes (core
    // columns 128 bytes apart) touch eight bank groups per warp.
    constexpr int NE = (G_ROWS * G_KC / 4) / G_CONSUMERS;   // 4 float4 per thread per chunk
    auto elem = [&](int k, int& row, int& c4) {
      row = (2 * warp + (k >> 1)) * 8 + (lane & 7);
      c4 = ((lane >> 3) + 4 * (k & 1) + row) & 7;
    };
    for (int li = 0; li < my_tiles && !bad; ++li) {
      int b, r0, ct;
      tile(li, b, r0, ct);
      // the pilot rows of this thread's two rows of the tile (null past R)
      const float2* prow[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int rg = r0 + (2 * warp + u) * 8 + (lane & 7);
        prow[u] = (LS && rg < R) ? pil + size_t(rg / M) * N : nullptr;
      }
      for (int c = 0; c < n_kc && !bad; ++c) {
        const int q = li * n_kc + c, s = q % G_STAGES, ab = q & 1;
        const int x0 = b * B + c * (G_KC / 2);
        // the pilots do not depend on the chunk's data: load them before waiting for it
        float4 pv[NE];
#pragma unroll
        for (int k = 0; k < NE; ++k) {
          int row, c4;
          elem(k, row, c4);
          const int sc = x0 + 2 * c4;
          pv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (LS && prow[k >> 1] && sc + 1 < N) pv[k] = __ldg(reinterpret_cast<const float4*>(prow[k >> 1] + sc));
        }
        if (*s_abort || !mbar_wait_bounded(&full[s], uint32_t(q / G_STAGES) & 1u)) {
          bad = true;
          break;
        }
        // A buffer ab was last read by the MMAs of chunk q - 2
        if (q >= 2 && !mbar_wait_bounded(&done[ab], uint32_t((q - 2) >> 1) & 1u)) {
          bad = true;
          break;
        }
        const float4* raw4 = reinterpret_cast<const float4*>(sRaw + s * G_RAW);
        unsigned char* ah = sA + ab * NP * G_A_PART;
        unsigned char* al = ah + G_A_PART;
#pragma unroll
        for (int k = 0; k < NE; ++k) {
          int row, c4;
          elem(k, row, c4);
          float4 v = raw4[row * 8 + c4];
          if (LS) {
            const int rg = r0 + row, sc = x0 + 2 * c4;
            const float4 p = pv[k];
            const float i0 = __fdividef(1.0f, fmaf(p.x, p.x, p.y * p.y));
            const float i1 = __fdividef(1.0f, fmaf(p.z, p.z, p.w * p.w));
            // rows past R and subcarriers past n_sc hold zeros (TMA fill): keep them zero
            v = (rg < R && sc + 1 < N)
                    ? make_float4(fmaf(v.x, p.x, v.y * p.y) * i0, fmaf(v.y, p.x, -v.x * p.y) * i0,
                                  fmaf(v.z, p.z, v.w * p.w) * i1, fmaf(v.w, p.z, -v.z * p.w) * i1)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          if constexpr (OP == G_TF32X3) {
            const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
            const int off = (row >> 3) * int(G_SBO) + c4 * 128 + (row & 7) * 16;
            *reinterpret_cast<float4*>(ah + off) = h;
            *reinterpret_cast<float4*>(al + off) = make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y),
                                                               tf32_rna(v.z - h.z), tf32_rna(v.w - h.w));
          } else {
            // four 16-bit reals: half of a 16-byte core row (eight reals)
            const int off = (row >> 3) * int(G_SBO) + (c4 >> 1) * 128 + (row & 7) * 16 + (c4 & 1) * 8;
            *reinterpret_cast<uint2*>(ah + off) =
                OP == G_FP16 ? make_uint2(pack_f16x2(v.x, v.y), pack_f16x2(v.z, v.w))
                             : make_uint2(pack_bf16x2(v.x, v.y), pack_bf16x2(v.z, v.w));
          }
        }
        fence_proxy_async_shared();              // the MMAs read what was written here
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&aready[ab]);
        mbar_arrive(&rawfree[s]);
        // the first chunk of group gg is handed over: drain the previous group meanwhile
        const int gg = li * gpt + c / G_DR;
        if (c % G_DR == 0 && gg >= 1 && !drain(gg - 1)) bad = true;
      }
    }
    if (!bad && my_tiles > 0 && !drain(my_tiles * gpt - 1)) bad = true;
    if (bad) give_up();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(TCOLS))
                 : "memory");
}

// ---------------------------------------------------------------- 16-bit forms, staged A
// The BF16 / FP16 forms round LS once per element: tcg_stage_kernel writes h_ls of every
// (block, 128-row tile, K chunk) as one 16-bit A chunk in the canonical K-major layout
// (the plan's staging buffer), so that the GEMM kernel below only copies and multiplies.
// Elements past the last row or subcarrier are zero; those of the next block that a last K
// chunk covers meet zero rows of W.  Chunks of the 16-bit forms are G16_KC = 64 reals (32
// subcarriers) wide: half as many commits and barrier round trips per MMA as 32.
constexpr int G16_KC = 64;                      // input reals per K chunk (32 subcarriers)
constexpr int G16_NS = 4;
constexpr int G16_THREADS = 192;
constexpr uint32_t G16_SBO = uint32_t(G16_KC * 2 / 16) * 128;   // 8-row group stride (bytes)
constexpr int G16_A_PART = G_ROWS * G16_KC * 2;                 // one A chunk (bytes)

template <int OP>
__global__ void __launch_bounds__(256) tcg_stage_kernel(const float2* __restrict__ y, const float2* __restrict__ pil,
                                                        unsigned char* __restrict__ a_tiles, int R, int M, int N,
                                                        int B, int n_kc, int n_rt) {
  // Thread -> one 16-byte core row (8 reals, 4 subcarriers) of a chunk row: loads of a warp
  // cover 4 chunk rows x 128 contiguous bytes, stores fill whole 32-byte sectors.
  constexpr int CC = G16_KC / 8;                     // core columns per chunk row
  const int c = blockIdx.x, rt = blockIdx.y, b = blockIdx.z;
  const int r0 = rt * G_ROWS, x0 = b * B + c * (G16_KC / 2);
  unsigned char* a = a_tiles + ((size_t(b) * n_rt + rt) * n_kc + c) * size_t(G16_A_PART);
  const int cc = threadIdx.x % CC;
#pragma unroll
  for (int k = 0; k < G_ROWS * CC / 256; ++k) {
    const int row = int(threadIdx.x) / CC + (256 / CC) * k, rg = r0 + row;
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {                    // two subcarriers per float4
      const int sc = x0 + 4 * cc + 2 * h;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rg < R && sc < N) {
        const float4 yv = __ldg(reinterpret_cast<const float4*>(y + size_t(rg) * N + sc));
        const float4 p = __ldg(reinterpret_cast<const float4*>(pil + size_t(rg / M) * N + sc));
        const float i0 = __fdividef(1.0f, fmaf(p.x, p.x, p.y * p.y));
        const float i1 = __fdividef(1.0f, fmaf(p.z, p.z, p.w * p.w));
        v = make_float4(fmaf(yv.x, p.x, yv.y * p.y) * i0, fmaf(yv.y, p.x, -yv.x * p.y) * i0,
                        fmaf(yv.z, p.z, yv.w * p.w) * i1, fmaf(yv.w, p.z, -yv.z * p.w) * i1);   // Eq. 9
      }
      w[2 * h] = OP == G_FP16 ? pack_f16x2(v.x, v.y) : pack_bf16x2(v.x, v.y);
      w[2 * h + 1] = OP == G_FP16 ? pack_f16x2(v.z, v.w) : pack_bf16x2(v.z, v.w);
    }
    const int off = (row >> 3) * int(G16_SBO) + cc * 128 + (row & 7) * 16;
    *reinterpret_cast<uint4*>(a + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// GEMM of the staged A chunks with W on tcgen05, 192 threads: four drain warps (warp w reads
// TMEM lanes 32 w .. 32 w + 31, i.e. rows), one MMA warp and one copy warp.  A ring of
// G16_NS stages holds each chunk's A (and W unless one column tile's W stays resident),
// brought by 1-D bulk copies; the MMA warp accumulates a tile's whole K into one of two FP32
// accumulators and commits the tile to an mbarrier, and the drain warps store that tile
// while the next one is multiplied into the other.  Persistent CTAs take runs of tiles as
// in lmmse_tcg_kernel; every wait is bounded.
// PAIR (streamed W): clusters of two CTAs take the two row tiles of a pair with the same
// column tile; each CTA brings half of every W chunk and multicasts it into both CTAs'
// stages, so W crosses from L2 once per pair.  A stage is refilled only when the MMAs of
// both CTAs are done with it (each commit arrives on both CTAs' barriers).  Both CTAs pass a
// cluster barrier after setting up their barriers and before leaving.

__device__ __forceinline__ void bulk_load_mc(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                             uint16_t cta_mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], "
      "%4;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar)), "h"(cta_mask)
      : "memory");
}

template <int NT, int OP, bool PAIR>
__global__ void __launch_bounds__(G16_THREADS, 1)
    lmmse_tcg16_kernel(const unsigned char* __restrict__ a_tiles, const unsigned char* __restrict__ w_tiles,
                       float2* __restrict__ out, int R, int N, int B, int n_kc, int n_rt, int n_rt_a, int n_ct,
                       int n_tiles, int w_resident, int* status) {
  static_assert(OP != G_TF32X3 && NT % 32 == 0 && NT <= 256, "16-bit forms, 32-column groups");
  constexpr int A_PART = G16_A_PART, W_PART = NT * G16_KC * 2;
  constexpr uint32_t G_SBO = G16_SBO;
  constexpr int KSTEPS = G16_KC * 2 / 32;               // MMAs per chunk (K = 16 each)
  constexpr int TCOLS = 2 * tmem_cols(NT);
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* pfull = reinterpret_cast<uint64_t*>(smem);   // [G16_NS] stage landed
  uint64_t* pdone = pfull + G16_NS;                      // [G16_NS] MMAs of the stage's chunk done
  uint64_t* tdone = pdone + G16_NS;                      // [2] a tile's MMAs done (per accumulator)
  uint64_t* drained = tdone + 2;                         // [2] accumulator read back
  uint64_t* wres = drained + 2;                          // resident W landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wres + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int stage_bytes = A_PART + (w_resident ? 0 : W_PART);
  unsigned char* ring = smem + 1024;                     // [G16_NS][A | W]
  unsigned char* sWres = ring + G16_NS * stage_bytes;    // resident W: [n_kc][W_PART]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // PAIR: a unit of work is a pair of row tiles (n_rt counts pairs); this CTA takes row tile
  // 2 rt + rank of each.  The staged A holds n_rt_a row tiles.
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const int unit = PAIR ? int(blockIdx.x >> 1) : int(blockIdx.x);
  const int n_units = PAIR ? int(gridDim.x >> 1) : int(gridDim.x);
  const int t_begin = int((long long)n_tiles * unit / n_units);
  const int my_tiles = int((long long)n_tiles * (unit + 1) / n_units) - t_begin;
  const int n_q = my_tiles * n_kc;
  auto tile = [&](int li, int& b, int& rt, int& ct) {
    const int t = t_begin + li;
    ct = t % n_ct;
    const int rest = t / n_ct;
    rt = rest % n_rt;
    b = rest / n_rt;
    if (PAIR) rt = 2 * rt + int(rank);
  };
  if (tid == 0) {
    for (int s = 0; s < G16_NS; ++s) {
      mbar_init(&pfull[s], 1);
      mbar_init(&pdone[s], PAIR ? 2 : 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tdone[i], 1);
      mbar_init(&drained[i], 128);
    }
    mbar_init(wres, 1);
    *s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(uint32_t(TCOLS))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (PAIR) cluster_sync_all();                          // the peer's barriers are set up
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&]() {
    *s_abort = 1;
    atomicExch(status, int(RAPRO_ERR_TIMEOUT));
  };
  if (warp == 5) {
    // ------------------------------------------------ copy warp
    if (lane == 0 && n_q > 0) {
      int issued = 0;
      bool bad = false;
      if (w_resident) {                         // one column tile: all of its W chunks, once
        mbar_arrive_expect_tx(wres, uint32_t(n_kc) * W_PART);
        bulk_load(sWres, w_tiles, uint32_t(n_kc) * W_PART, wres);
      }
      for (int q = 0; q < n_q && !bad; ++q) {
        const int li = q / n_kc, c = q - li * n_kc, s = q % G16_NS;
        int b, rt, ct;
        tile(li, b, rt, ct);
        // stage s was last read by the MMAs of chunk q - G16_NS
        if (q >= G16_NS && !mbar_wait_bounded(&pdone[s], uint32_t(q / G16_NS - 1) & 1u)) {
          bad = true;
          break;
        }
        unsigned char* st = ring + s * stage_bytes;
        mbar_arrive_expect_tx(&pfull[s], uint32_t(stage_bytes));
        bulk_load(st, a_tiles + ((size_t(b) * n_rt_a + rt) * n_kc + c) * A_PART, A_PART, &pfull[s]);
        const unsigned char* wsrc = w_tiles + (size_t(ct) * n_kc + c) * W_PART;
        if (PAIR)          // this CTA's half of the chunk's W rows, into both CTAs' stage s
          bulk_load_mc(st + A_PART + rank * (W_PART / 2), wsrc + rank * (W_PART / 2), W_PART / 2, &pfull[s], 0x3);
        else if (!w_resident)
          bulk_load(st + A_PART, wsrc, W_PART, &pfull[s]);
        ++issued;
        if (*s_abort) bad = true;
      }
      // Let the copies in flight land before the CTA moves on (all consumed on the normal path).
      for (int s = 0; s < G16_NS && s < issued; ++s)
        (void)mbar_wait_bounded(&pfull[s], uint32_t((issued - 1 - s) / G16_NS) & 1u);
      if (w_resident) (void)mbar_wait_bounded(wres, 0u);
      if (bad) give_up();
    }
  } else if (warp == 4) {
    // ------------------------------------------------ MMA warp: one thread issues
    if (lane == 0 && n_q > 0) {
      int issued = 0;
      bool bad = false;
      if (w_resident && !mbar_wait_bounded(wres, 0u)) bad = true;
      for (int q = 0; q < n_q && !bad; ++q) {
        const int li = q / n_kc, c = q - li * n_kc, s = q % G16_NS;
        // accumulator li & 1 was last drained for tile li - 2
        if (c == 0 && li >= 2 && !mbar_wait_bounded(&drained[li & 1], uint32_t((li - 2) >> 1) & 1u)) {
          bad = true;
          break;
        }
        if (!mbar_wait_bounded(&pfull[s], uint32_t(q / G16_NS) & 1u) || *s_abort) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char* a = ring + s * stage_bytes;
        const unsigned char* w = w_resident ? sWres + size_t(c) * W_PART : a + A_PART;
        const uint32_t d = tmem + uint32_t((li & 1) * tmem_cols(NT));
#pragma unroll
        for (int ks = 0; ks < KSTEPS; ++ks)
          mma_g<NT, OP>(d, smem_desc_kmajor(a + ks * 256, 128, G_SBO), smem_desc_kmajor(w + ks * 256, 128, G_SBO),
                        c > 0 || ks > 0);
        if (PAIR)          // stage s is free once both CTAs' MMAs are done with it
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                  smem_u32(&pdone[s])),
              "h"(uint16_t(0x3))
              : "memory");
        else
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&pdone[s]))
                       : "memory");
        if (c == n_kc - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&tdone[li & 1]))
                       : "memory");
        ++issued;
      }
      // The tensor cores finish in order: the last chunk done means TMEM may be freed.
      if (issued > 0)
        (void)mbar_wait_bounded(&pdone[(issued - 1) % G16_NS], uint32_t((issued - 1) / G16_NS) & 1u);
      if (bad) give_up();
    }
  } else {
    // ------------------------------------------------ drain warps: TMEM -> output
    for (int li = 0; li < my_tiles; ++li) {
      if (*s_abort || !mbar_wait_bounded(&tdone[li & 1], uint32_t(li >> 1) & 1u)) {
        give_up();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int b, rt, ct;
      tile(li, b, rt, ct);
      const int row = rt * G_ROWS + 32 * warp + lane;
#pragma unroll 1
      for (int g = 0; g < NT / 32; ++g) {
        uint32_t v[32];
        tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t((li & 1) * tmem_cols(NT) + 32 * g), v);
        const int j0 = (ct * NT + 32 * g) >> 1;       // first complex output of the group
        if (row < R) {
          // pairs of outputs as 16-byte stores (row * N + b * B + j0 is even; so is B)
          float4* o = reinterpret_cast<float4*>(out + size_t(row) * N + size_t(b) * B + j0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j0 + 2 * j < B)
              o[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&drained[li & 1]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (PAIR) cluster_sync_all();                          // no copy or arrival still bound for this CTA
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(TCOLS))
                 : "memory");
}

template <int NT, int OP>
constexpr size_t tcg16_smem_bytes(int n_kc, bool w_resident) {
  return 1024 + size_t(G16_NS) * (G16_A_PART + (w_resident ? 0 : NT * G16_KC * 2)) +
         (w_resident ? size_t(n_kc) * NT * G16_KC * 2 : 0);
}

// ------------------------------------------------------------------------------ host
// Output reals per tile: 96 or 128, and 256 for the 16-bit forms from B = 128 (each converted
// A chunk then feeds twice the MMA work).
static int tcg_nt(int B, int op) { return 2 * B <= 96 ? 96 : (op != G_TF32X3 && B >= 128 ? 256 : 128); }

template <int NT, int OP>
static size_t tcg_smem_bytes(int w_chunks) {
  return 1024 + 2 * size_t(g_parts(OP)) * g_a_part(OP) + size_t(w_chunks) * g_parts(OP) * NT * G_KC * g_elt(OP) +
         size_t(G_STAGES) * G_RAW;
}

static int tcg_op(const Plan& pl) {
  return pl.p.precision == RAPRO_PREC_BF16 ? G_BF16 : pl.p.precision == RAPRO_PREC_FP16 ? G_FP16 : G_TF32X3;
}

constexpr size_t kTcgSmemMax = 232448;   // 227 KB, the per-CTA limit


// Blocks up to 2048 subcarriers (W tiles of up to 128 MB).  The drained accumulation keeps
// the error at that of a K = 128 sum (measured at n_sc = 1200, B = 1200: 1.6e-5 relative
// with one accumulator over all of K = 2400, against the 1e-5 bar).
constexpr int kTcgMaxBlock = 2048;

bool lmmse_tcg_shape_ok(const Plan& pl) {
  const long long rows = (long long)pl.T * pl.p.K * pl.p.M;
  return !pl.comb && pl.B > 16 && pl.B <= kTcgMaxBlock && pl.B % 2 == 0 && pl.tail == 0 &&
         rows < (1ll << 31) && pl.p.n_sc / pl.B <= 65535;
}

// Wr (2B x 2B reals) cut into tiles of NT output reals x chunks of 32 input reals, each
// chunk TF32 hi then lo (or one BF16 / FP16 part) in the canonical K-major layout, tiles one
// after the other.
void build_lmmse_tcg_weights(const Plan& pl, std::vector<unsigned char>& out) {
  const int op = tcg_op(pl), elt = g_elt(op), np = g_parts(op);
  const int KC = op == G_TF32X3 ? G_KC : G16_KC;   // K chunk of the kernel that reads the tiles
  const uint32_t sbo = uint32_t(KC * elt / 16) * 128;
  const int B = pl.B, NT = tcg_nt(B, op), K2 = 2 * B;
  const int n_nt = (K2 + NT - 1) / NT, n_kc = (K2 + KC - 1) / KC;
  const size_t part = size_t(NT) * KC * elt;
  out.assign(size_t(n_nt) * n_kc * np * part, 0);
  for (int t = 0; t < n_nt; ++t)
    for (int c = 0; c < n_kc; ++c) {
      unsigned char* base = out.data() + (size_t(t) * n_kc + c) * np * part;
      for (int nn = 0; nn < NT; ++nn)
        for (int kk = 0; kk < KC; ++kk) {
          const int n = t * NT + nn, k = c * KC + kk;
          if (n >= K2 || k >= K2) continue;
          const float2 w = pl.w_main[size_t(n >> 1) * B + (k >> 1)];
          const float vals[2][2] = {{w.x, -w.y}, {w.y, w.x}};   // [out re/im][in re/im]
          const float f = vals[n & 1][k & 1];
          const int ce = 16 / elt;                        // reals per 16-byte core row
          const size_t off = size_t((nn >> 3) * sbo + (kk / ce) * 128 + (nn & 7) * 16 + (kk % ce) * elt);
          if (op == G_TF32X3) {
            const float h = tf32_round_host(f), l = tf32_round_host(f - h);
            std::memcpy(base + off, &h, 4);
            std::memcpy(base + part + off, &l, 4);
          } else {
            const uint16_t v16 = op == G_FP16 ? f16_round_host(f) : bf16_round_host(f);
            std::memcpy(base + off, &v16, 2);
          }
        }
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 tcg_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool lmmse_tcg_ok(const Plan& pl, const float2* x, const float2* out) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(out);
  return pl.d_w_tcg != nullptr && (a & 15) == 0 && lmmse_tcg_shape_ok(pl) && tcg_encode() != nullptr &&
         (tcg_op(pl) == G_TF32X3 || pl.d_a_tcg != nullptr);
}

// The 16-bit forms' staged A operand: [blocks][row tiles][K chunks] canonical chunks (0 for
// the TF32 form and other shapes).
size_t lmmse_tcg_stage_bytes(const Plan& pl) {
  const int op = tcg_op(pl);
  if (op == G_TF32X3 || !lmmse_tcg_shape_ok(pl)) return 0;
  const long long R = (long long)pl.T * pl.p.K * pl.p.M;
  const long long n_rt_a = 2 * ((R + 2 * G_ROWS - 1) / (2 * G_ROWS)), n_kc = (2 * pl.B + G16_KC - 1) / G16_KC;
  return size_t(pl.p.n_sc / pl.B) * size_t(n_rt_a) * size_t(n_kc) * size_t(G16_A_PART);
}

template <int NT, int OP>
static cudaError_t launch_tcg16(const Plan& pl, const float2* y, const float2* pil, float2* out, cudaStream_t st) {
  if (!pil || !pl.d_a_tcg) return cudaErrorNotSupported;   // the 16-bit forms take the LS-fused input only
  const int B = pl.B, N = pl.p.n_sc, M = pl.p.M, R = pl.T * pl.p.K * pl.p.M;
  const int n_nt = (2 * B + NT - 1) / NT, n_kc = (2 * B + G16_KC - 1) / G16_KC, n_rt = (R + G_ROWS - 1) / G_ROWS;
  const int n_rt_a = 2 * ((n_rt + 1) / 2), nb = N / B;   // staged row tiles: an even count
  if (n_rt_a > 65535) return cudaErrorInvalidValue;
  unsigned char* a = static_cast<unsigned char*>(pl.d_a_tcg);
  const unsigned char* w = static_cast<const unsigned char*>(pl.d_w_tcg);
  tcg_stage_kernel<OP><<<dim3(n_kc, n_rt_a, nb), 256, 0, st>>>(y, pil, a, R, M, N, B, n_kc, n_rt_a);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool w_resident = n_nt == 1 && tcg16_smem_bytes<NT, OP>(n_kc, true) <= kTcgSmemMax;
  if (w_resident) {                                     // one column tile: no W to share
    const long long tiles = (long long)n_rt * nb;
    if (tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    const int n_tiles = int(tiles), grid = std::min(n_tiles, sms);   // one CTA per SM (shared memory, TMEM)
    lmmse_tcg16_kernel<NT, OP, false><<<grid, G16_THREADS, tcg16_smem_bytes<NT, OP>(n_kc, true), st>>>(
        a, w, out, R, N, B, n_kc, n_rt, n_rt_a, n_nt, n_tiles, 1, pl.d_status);
    return cudaGetLastError();
  }
  // CTA pairs over pairs of row tiles
  const long long tiles = (long long)(n_rt_a / 2) * n_nt * nb;
  if (tiles >= (1ll << 30)) return cudaErrorInvalidValue;
  const int n_tiles = int(tiles);
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(G16_THREADS, 1, 1);
  cfg.dynamicSmemBytes = tcg16_smem_bytes<NT, OP>(n_kc, false);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // as many pairs as can be resident at once (pairs sit on two SMs of one GPC)
  cfg.gridDim = dim3(2 * std::max(1, std::min(n_tiles, sms / 2)), 1, 1);
  int fit = 0;
  if (cudaOccupancyMaxActiveClusters(&fit, lmmse_tcg16_kernel<NT, OP, true>, &cfg) != cudaSuccess) fit = 0;
  cfg.gridDim = dim3(2 * std::max(1, std::min({n_tiles, sms / 2, fit > 0 ? fit : sms / 2})), 1, 1);
  return cudaLaunchKernelEx(&cfg, lmmse_tcg16_kernel<NT, OP, true>, static_cast<const unsigned char*>(a), w, out, R,
                            N, B, n_kc, n_rt_a / 2, n_rt_a, n_nt, n_tiles, 0, pl.d_status);
}

template <int NT, int OP>
static cudaError_t launch_tcg_nt(const Plan& pl, const float2* x, const float2* pil, float2* out, cudaStream_t st) {
  const int B = pl.B, N = pl.p.n_sc, M = pl.p.M, R = pl.T * pl.p.K * pl.p.M;
  const int n_nt = (2 * B + NT - 1) / NT, n_kc = (2 * B + G_KC - 1) / G_KC;
  // 2-D map over x [R][N] complex64 with boxes of 16 subcarriers x 128 rows.
  CUtensorMap map;
  cuuint64_t dims[2] = {cuuint64_t(N), cuuint64_t(R)};
  cuuint64_t strides[1] = {cuuint64_t(N) * 8};
  cuuint32_t box[2] = {cuuint32_t(G_KC / 2), cuuint32_t(G_ROWS)};
  cuuint32_t es[2] = {1, 1};
  if (tcg_encode()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<float2*>(x), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int n_rt = (R + G_ROWS - 1) / G_ROWS;
  const long long tiles = (long long)n_rt * n_nt * (N / B);
  if (tiles >= (1ll << 31)) return cudaErrorInvalidValue;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = int(tiles), grid = std::min(n_tiles, sms);   // one CTA per SM (shared memory)
  const int w_resident = n_nt == 1 && n_kc > 2 && tcg_smem_bytes<NT, OP>(n_kc) <= kTcgSmemMax ? 1 : 0;
  const size_t smem = tcg_smem_bytes<NT, OP>(w_resident ? n_kc : 2);
  const unsigned char* w = static_cast<const unsigned char*>(pl.d_w_tcg);
  if (pil)
    lmmse_tcg_kernel<NT, true, OP><<<grid, G_THREADS, smem, st>>>(map, pil, out, w, R, M, N, B, n_kc, n_rt, n_nt,
                                                                  n_tiles, w_resident, pl.d_status);
  else if constexpr (OP == G_TF32X3)
    lmmse_tcg_kernel<NT, false, OP><<<grid, G_THREADS, smem, st>>>(map, pil, out, w, R, M, N, B, n_kc, n_rt,
                                                                   n_nt, n_tiles, w_resident, pl.d_status);
  else
    return cudaErrorNotSupported;                    // the 16-bit forms take the LS-fused input only
  return cudaGetLastError();
}

cudaError_t launch_lmmse_tcg(const Plan& pl, const float2* x, const float2* pil, float2* out, cudaStream_t st) {
  const int op = tcg_op(pl), nt = tcg_nt(pl.B, op);
  switch (op) {
    case G_BF16:
      return nt == 96    ? launch_tcg16<96, G_BF16>(pl, x, pil, out, st)
             : nt == 128 ? launch_tcg16<128, G_BF16>(pl, x, pil, out, st)
                         : launch_tcg16<256, G_BF16>(pl, x, pil, out, st);
    case G_FP16:
      return nt == 96    ? launch_tcg16<96, G_FP16>(pl, x, pil, out, st)
             : nt == 128 ? launch_tcg16<128, G_FP16>(pl, x, pil, out, st)
                         : launch_tcg16<256, G_FP16>(pl, x, pil, out, st);
    default:
      return nt == 96 ? launch_tcg_nt<96, G_TF32X3>(pl, x, pil, out, st) : launch_tcg_nt<128, G_TF32X3>(pl, x, pil, out, st);
  }
}

template <int OP>
static cudaError_t set_tcg16_smem(int bytes) {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(lmmse_tcg16_kernel<96, OP, false>, A, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg16_kernel<128, OP, false>, A, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg16_kernel<256, OP, false>, A, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg16_kernel<96, OP, true>, A, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg16_kernel<128, OP, true>, A, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg16_kernel<256, OP, true>, A, bytes);
  return e;
}

cudaError_t prepare_lmmse_tcg(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int S = int(kTcgSmemMax);
    cudaError_t e = cudaFuncSetAttribute(lmmse_tcg_kernel<96, true, G_TF32X3>, A, S);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg_kernel<96, false, G_TF32X3>, A, S);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg_kernel<128, true, G_TF32X3>, A, S);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_tcg_kernel<128, false, G_TF32X3>, A, S);
    if (e == cudaSuccess) e = set_tcg16_smem<G_BF16>(S);
    if (e == cudaSuccess) e = set_tcg16_smem<G_FP16>(S);
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
