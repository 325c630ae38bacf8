// Gram matrix and matched filter of the MMSE detector (Eq. 22) on the 5th-generation tensor
// cores with 16-bit operands (the precision form's detector half):
//   A[t][k] = H_k^H H_k + sigma2 I   and   z[t][k] = H_k^H Y_k
// per (slot t, subcarrier k), H_k = h[t][:, :, k] (K users x M antennas), Y_k the slot's D
// data symbols at subcarrier k.
//
// Real embedding.  With the contraction index running over (antenna m, re/im) interleaved,
// a user row u_s = (Re h_s,0, Im h_s,0, Re h_s,1, ...) and, for every column c of [H | Y]
// (user or data symbol, vector v_c over the antennas), the two operand columns
//   (Re v_c,0, Im v_c,0, ...)   and   (Im v_c,0, -Re v_c,0, ...)
// give u_s . col = Re(h_s^H v_c) and Im(h_s^H v_c).  So one real GEMM per subcarrier,
// K x 2M times 2M x 2C (C = K + D), yields the K x C complex block [A - sigma2 I | z].
//
// Packing.  A subcarrier's block is tiny, so 8 subcarriers share one MMA tile: row
// 16 j + s holds user s of subcarrier j of the tile (users padded to 16), and the columns of
// subcarriers 0-3 and 4-7 form two N-tiles of 4 x 2C columns (padded to a multiple of 16),
// one accumulator each in tensor memory.  The MMA also forms the products of one
// subcarrier's users with another's columns; only the diagonal blocks are read back, so the
// tensor cores do about a tenth useful work (K = 12, D = 6: 12 of every 128 rows).
//
// One CTA per (slot, 8 subcarriers), four roles ordered by mbarriers only:
//  * a TMA warp streams 8-antenna chunks (8 subcarriers x 8 antennas x K users of h and x D
//    symbols of y, complex64) into a ring of FP32 stages;
//  * eight converter warps round each chunk to BF16 (or FP16) into the canonical K-major
//    layout of a ring of operand buffers (8-row x 16-byte core matrices); one chunk is one
//    K step (8 antennas x re/im = 16 values) of the MMA;
//  * one thread issues the two MMAs of a chunk (M = 128, N = 4 x 2C, K = 16, FP32
//    accumulation) and commits them to the operand buffer's free barrier;
//  * after the last chunk converter warps 0-3 read their tensor-memory lanes back (lane =
//    row), keep their own subcarrier's columns, add sigma2 on the diagonal and write
//    G[t][k][s][c] = (A | z)[s][c].
#include <algorithm>
#include <mutex>

#include "rapro_internal.h"
#include "rapro_ptx.cuh"

namespace rapro {

namespace {

constexpr int GT_SC = 8;                    // subcarriers per tile
constexpr int GT_ROWS = 128;                // MMA M: 8 subcarriers x 16 user rows
constexpr int GT_FST = 8;                   // FP32 stage ring
constexpr int GT_BST = 3;                   // 16-bit operand ring
constexpr int GT_CONV = 256;                // converter threads (the first 128 also read back)
constexpr int GT_THREADS = GT_CONV + 64;    // + MMA warp + TMA warp
constexpr int GT_TMEM_COLS = 512;
constexpr int GT_A_BYTES = GT_ROWS * 32;    // 128 rows x 16 values x 2 bytes
constexpr int GT_MAX_C = RAPRO_MAX_USERS + RAPRO_MAX_DATA_PER_SLOT;

enum { GOP_BF16 = 0, GOP_FP16 = 1 };

struct GramParams {
  int T, K, M, N, D, C;    // C = K + D complex columns
  int NT;                  // columns of one N-tile: 4 x 2C padded to a multiple of 16
  int nchunks;             // 8-antenna chunks
  float sigma2;
  float2* G;               // [T][N][K][C]
  int* status;
};

__host__ __device__ constexpr int gram_nt(int C) { return (8 * C + 15) / 16 * 16; }
__host__ __device__ constexpr size_t gram_fstage_bytes(int C) { return size_t(C) * 8 * GT_SC * sizeof(float2); }
__host__ __device__ constexpr size_t gram_bstage_bytes(int NT) { return size_t(GT_A_BYTES) + 2 * size_t(NT) * 32; }
size_t gram_smem_bytes(int C) {
  return 1024 + GT_FST * gram_fstage_bytes(C) + GT_BST * gram_bstage_bytes(gram_nt(C));
}

// Byte offset of row r, core column kc (0 or 1) in a canonical K-major operand of 16 values
// per row: 8-row groups of two 128-byte core matrices.
__device__ __forceinline__ int canon_off(int r, int kc) { return (r >> 3) * 256 + kc * 128 + (r & 7) * 16; }

template <int OP>
__device__ __forceinline__ uint32_t pk(float lo, float hi) {
  if constexpr (OP == GOP_FP16) return pack_f16x2(lo, hi);
  else return pack_bf16x2(lo, hi);
}

template <int OP>
__device__ __forceinline__ void gram_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc ? 1 : 0)
      : "memory");
}

// 16 consecutive columns of this warp's 32 TMEM lanes, waited for.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

template <int OP>
__global__ void __launch_bounds__(GT_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap map_h, const __grid_constant__ CUtensorMap map_y,
                   const __grid_constant__ GramParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* ffull = reinterpret_cast<uint64_t*>(smem);      // [GT_FST] chunk landed
  uint64_t* ffree = ffull + GT_FST;                         // [GT_FST] chunk converted
  uint64_t* bready = ffree + GT_FST;                        // [GT_BST] operands written
  uint64_t* bfree = bready + GT_BST;                        // [GT_BST] MMAs done reading
  uint64_t* mdone = bfree + GT_BST;                         // every MMA finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int C = P.C, K = P.K, D = P.D, NT = P.NT;
  const size_t fbytes = gram_fstage_bytes(C), bbytes = gram_bstage_bytes(NT);
  unsigned char* fring = smem + 1024;
  unsigned char* bring = fring + GT_FST * fbytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t = blockIdx.y, sc0 = blockIdx.x * GT_SC;

  // Operand rows that no chunk writes (users K..15 of A, columns past 4 x 2C of each
  // N-tile) stay zero: clear every operand buffer once.
  for (int e = tid; e < int(GT_BST * bbytes / 16); e += GT_THREADS)
    reinterpret_cast<uint4*>(bring)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int s = 0; s < GT_FST; ++s) {
      mbar_init(&ffull[s], 1);
      mbar_init(&ffree[s], GT_CONV);
    }
    for (int b = 0; b < GT_BST; ++b) {
      mbar_init(&bready[b], GT_CONV);
      mbar_init(&bfree[b], 1);
    }
    mbar_init(mdone, 1);
    *s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(GT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async_shared();          // the cleared operand buffers, before any MMA reads them
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&]() {
    *s_abort = 1;
    atomicExch(P.status, int(RAPRO_ERR_TIMEOUT));
  };

  if (warp == GT_CONV / 32 + 1) {
    // ------------------------------------------------------------ TMA warp
    if (lane == 0) {
      prefetch_tensormap(&map_h);
      prefetch_tensormap(&map_y);
      const uint32_t tx = uint32_t(fbytes);
      int issued = 0;
      bool bad = false;
      for (int c = 0; c < P.nchunks; ++c) {
        const int s = c % GT_FST;
        if (c >= GT_FST && (!mbar_wait_bounded(&ffree[s], uint32_t(c / GT_FST - 1) & 1u) || *s_abort)) {
          bad = true;
          break;
        }
        float2* st = reinterpret_cast<float2*>(fring + s * fbytes);
        mbar_arrive_expect_tx(&ffull[s], tx);
        tma_load_3d(st, &map_h, &ffull[s], sc0, c * 8, t * K);
        tma_load_3d(st + K * 8 * GT_SC, &map_y, &ffull[s], sc0, c * 8, t * D);
        ++issued;
      }
      // Every issued load lands before the CTA exits: load j of stage s completes phase j / GT_FST.
      for (int s = 0; s < GT_FST && s < issued; ++s)
        (void)mbar_wait_bounded(&ffull[s], uint32_t((issued - 1 - s) / GT_FST) & 1u);
      if (bad) give_up();
    }
  } else if (warp == GT_CONV / 32) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      // D = F32, A = B = BF16 (1) or FP16 (0), both K-major, N = NT, M = 128.
      const uint32_t fmt = OP == GOP_FP16 ? 0u : 1u;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(NT >> 3) << 17) |
                             (uint32_t(GT_ROWS >> 4) << 24);
      int issued = 0;
      bool bad = false;
      for (int c = 0; c < P.nchunks; ++c) {
        const int b = c % GT_BST;
        if (!mbar_wait_bounded(&bready[b], uint32_t(c / GT_BST) & 1u) || *s_abort) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char* ba = bring + b * bbytes;
        const unsigned char* bb = ba + GT_A_BYTES;
        const uint64_t da = smem_desc_kmajor(ba, 128, 256);
#pragma unroll
        for (int q = 0; q < 2; ++q)
          gram_mma<OP>(tmem + uint32_t(q * NT), da, smem_desc_kmajor(bb + q * NT * 32, 128, 256), idesc, c > 0);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bfree[b]))
                     : "memory");
        ++issued;
      }
      // Completes once every MMA issued above has finished (also on the abort path, so
      // that tensor memory is freed only after them).
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mdone))
                   : "memory");
      if (bad) give_up();
    }
  } else {
    // ------------------------------------------------------------ converters
    bool bad = false;
    for (int c = 0; c < P.nchunks; ++c) {
      const int s = c % GT_FST, b = c % GT_BST;
      if (*s_abort || !mbar_wait_bounded(&ffull[s], uint32_t(c / GT_FST) & 1u) ||
          (c >= GT_BST && !mbar_wait_bounded(&bfree[b], uint32_t(c / GT_BST - 1) & 1u))) {
        bad = true;
        break;
      }
      const float2* st = reinterpret_cast<const float2*>(fring + s * fbytes);   // [C][8 m][8 sc]
      unsigned char* ba = bring + b * bbytes;
      unsigned char* bb = ba + GT_A_BYTES;
      for (int it = tid; it < GT_SC * C; it += GT_CONV) {
        const int j = it & (GT_SC - 1), cc = it >> 3;   // subcarrier of the tile, column of [H | Y]
        float2 v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = st[(cc * 8 + m) * GT_SC + j];
        uint4 p0[2], p1[2];   // (re, im) pairs and (im, -re) pairs, 4 antennas per core row
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          p0[h] = make_uint4(pk<OP>(v[4 * h].x, v[4 * h].y), pk<OP>(v[4 * h + 1].x, v[4 * h + 1].y),
                             pk<OP>(v[4 * h + 2].x, v[4 * h + 2].y), pk<OP>(v[4 * h + 3].x, v[4 * h + 3].y));
          p1[h] = make_uint4(pk<OP>(v[4 * h].y, -v[4 * h].x), pk<OP>(v[4 * h + 1].y, -v[4 * h + 1].x),
                             pk<OP>(v[4 * h + 2].y, -v[4 * h + 2].x), pk<OP>(v[4 * h + 3].y, -v[4 * h + 3].x));
        }
        const int q = j >> 2, n0 = (j & 3) * 2 * C + 2 * cc;          // N-tile, column within it
        unsigned char* bq = bb + q * NT * 32;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          *reinterpret_cast<uint4*>(bq + canon_off(n0, h)) = p0[h];
          *reinterpret_cast<uint4*>(bq + canon_off(n0 + 1, h)) = p1[h];
          if (cc < K) *reinterpret_cast<uint4*>(ba + canon_off(j * 16 + cc, h)) = p0[h];
        }
      }
      fence_proxy_async_shared();          // the MMAs read what was written here
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&bready[b]);
      mbar_arrive(&ffree[s]);
    }
    if (bad) give_up();
    // ------------------------------------------------------------ read-back
    if (warp >= 4) {
      // warps 4-7 only convert: the 128 TMEM lanes belong to warps 0-3
    } else if (!bad && mbar_wait_bounded(mdone, 0u) && !*s_abort) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // Warp w holds rows 32w..32w+31: users of subcarriers 2w (lanes 0-15) and 2w+1.
      const int j = 2 * warp + (lane >> 4), s_user = lane & 15;
      const int q = warp >> 1;
      const int col0 = q * NT + ((2 * warp) & 3) * 2 * C;   // subcarrier 2w's first column
      const int sc = sc0 + j;
      const bool live = s_user < K && sc < P.N;
      float2* g = P.G + ((size_t(t) * P.N + (live ? sc : 0)) * K + (live ? s_user : 0)) * C;
      const uint32_t lane_base = tmem + (uint32_t(32 * warp) << 16);
      for (int c16 = 0; c16 < 2 * C; c16 += 16) {
        uint32_t u0[16], u1[16];
        tmem_ld16(lane_base + uint32_t(col0 + c16), u0);            // subcarrier 2w's columns
        tmem_ld16(lane_base + uint32_t(col0 + 2 * C + c16), u1);    // subcarrier 2w + 1's
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
          const int col = c16 + e, cc = col >> 1;
          if (live && col < 2 * C) {
            float2 val = (lane < 16) ? make_float2(__uint_as_float(u0[e]), __uint_as_float(u0[e + 1]))
                                     : make_float2(__uint_as_float(u1[e]), __uint_as_float(u1[e + 1]));
            if (cc == s_user) val.x += P.sigma2;
            g[cc] = val;
          }
        }
      }
    } else if (!bad) {
      give_up();
    }
  }
  // Tensor memory is freed only after every MMA has finished (mdone).
  if (tid == 0) (void)mbar_wait_bounded(mdone, 0u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT_TMEM_COLS) : "memory");
}

bool gram_tc_ok(const Plan& pl, const void* h, const void* y) {
  const bool aligned = ((reinterpret_cast<uintptr_t>(h) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  return aligned && !pl.comb && pl.p.n_sc % 2 == 0 && pl.p.K <= RAPRO_MAX_USERS && pl.D <= RAPRO_MAX_DATA_PER_SLOT;
}

cudaError_t launch_gram_tc(const Plan& pl, const float2* h, const float2* y, float2* G, bool fp16,
                           cudaStream_t st) {
  GramParams P{};
  P.T = pl.T; P.K = pl.p.K; P.M = pl.p.M; P.N = pl.p.n_sc; P.D = pl.D;
  P.C = P.K + P.D;
  P.NT = gram_nt(P.C);
  P.nchunks = (P.M + 7) / 8;
  P.sigma2 = float(pl.p.sigma2);
  P.G = G;
  P.status = pl.d_status;
  CUtensorMap mh, my;
  if (!encode_cx_map(&mh, h, P.N, P.M, P.T * P.K, P.K, GT_SC) ||
      !encode_cx_map(&my, y, P.N, P.M, P.T * P.D, P.D, GT_SC))
    return cudaErrorInvalidValue;
  const dim3 grid((P.N + GT_SC - 1) / GT_SC, P.T), block(GT_THREADS);
  const size_t smem = gram_smem_bytes(P.C);
  if (fp16) gram_tc_kernel<GOP_FP16><<<grid, block, smem, st>>>(mh, my, P);
  else gram_tc_kernel<GOP_BF16><<<grid, block, smem, st>>>(mh, my, P);
  return cudaGetLastError();
}

cudaError_t prepare_gram_tc(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const int smem = int(gram_smem_bytes(GT_MAX_C));
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<GOP_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gram_tc_kernel<GOP_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
