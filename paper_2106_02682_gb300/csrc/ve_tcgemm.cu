// ve_tcgemm.cu -- batched 256 x 256 x 256 products on the fifth-generation tensor cores, the
// GEMM-shaped part of the float32 PSD projections of 256 x 256 marginals (Eq. (rhoijTildeUpdate)
// and the per-wavevector step of Algorithm 6 of Khoo & Lindsey, arXiv:2106.02682): forming
// V^H C V from the previous eigenvectors, updating them, and the reconstruction V M V^H.
//
// Operands are "split" float32 matrices: each real plane p of a matrix is stored as two planes,
// hi = p rounded down to tf32 (the 10 significand bits the tensor core reads) and lo = p - hi
// (exact), and a product P Q^T is taken as Phi Qhi^T + Phi Qlo^T + Plo Qhi^T in kind::tf32 MMAs
// with float32 accumulation in tensor memory -- float32-level accuracy (~2^-21 relative per
// product term) at the tf32 rate.  Complex matrices carry planes (re hi, re lo, im hi, im lo).
//
// Storage of one 256 x 256 plane, "KC4": element (r, k) at ((k / 4) * 256 + r) * 4 + k % 4 --
// every 4 consecutive k of a row form one 16-byte chunk, and the chunks of consecutive rows are
// adjacent.  A TMA box of 4 x R x 4 over (k % 4, r, k / 4) then lands in shared memory exactly in
// the tensor core's no-swizzle K-major layout (8-row x 16-byte core matrices, 128 contiguous
// bytes each), and a thread reading one row's chunk as a float4 is coalesced with its
// neighbours.
//
// Kernel: one CTA per SM, persistent over (matrix, half, column group) tiles of 128 output rows.
// Warp 0 issues the TMA loads of 16-wide K slices into a ring of stages, warp 1 allocates tensor
// memory and issues the MMAs from one thread into one of two accumulators where they fit, and
// warps 2-9 read the other accumulator back (tcgen05.ld) meanwhile and write the split result,
// normal and/or transposed.  Every wait is bounded (ve_tc.cuh).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "../../include/ve.h"
#include "ve_internal.h"
#include "ve_tc.cuh"

namespace ve {

namespace {

using namespace tc;

// ROT: the right factor is a block rotation R (see tc_rot256), stored compactly: per pair its
// 32 x 32 block (rows: the pair's 32 output columns, K: the pair's 32 indices).  A stage's K slice
// is one block of the pair, and one 32-row box per plane feeds N = 32 MMAs into the accumulator
// slots of both output blocks.
//
// A tile is (matrix, 128-row half, column group): NCG column groups of TN output columns.  Its
// accumulator (re, and im when complex) takes ACC tensor-memory columns, and NBUF = 512 / ACC
// accumulators are in flight, so that the epilogue of one tile overlaps the MMAs of the next.
// A full product has one column group; a complex rotation has two (4 pairs, 8 column blocks
// each), which makes its accumulator half as wide and lets it double-buffer too.
//
// RAW (the rotations): x arrives plain -- NPX float32 planes, re (and im) -- and four converter
// warps split each landed K slice into the hi / lo planes the MMAs read, in shared memory.  A
// stage then holds [split x | y | raw x]; the TMA fills y and raw x, the converters split x.
template <bool CPLX, bool ROT = false>
struct TcCfg {
  static constexpr int NPL = CPLX ? 4 : 2;            // planes of a split matrix
  static constexpr int NPX = CPLX ? 2 : 1;            // planes of a plain matrix
  static constexpr bool RAW = ROT;                    // x plain, split in the kernel
  static constexpr int KS = 16;                       // K elements per stage
  static constexpr int XB = 128 * KS * 4;             // bytes of one X plane slice (128 rows)
  static constexpr int YR = ROT ? 2 * TC_BJ_BS : 256;  // rows of one Y plane slice
  static constexpr int YB = YR * KS * 4;               // bytes of one Y plane slice
  static constexpr int NYS = 1;                        // Y slices per plane and stage
  static constexpr int RAWOFF = NPL * (XB + NYS * YB);  // raw x within a stage
  static constexpr int STAGE_BYTES = RAWOFF + (RAW ? NPX * XB : 0);
  static constexpr int TX_BYTES = (RAW ? NPX : NPL) * XB + NPL * NYS * YB;  // loaded by the TMA
  static constexpr int STAGES = RAW ? (CPLX ? 3 : 4) : (CPLX ? 2 : 4);
  static constexpr int NCG = (ROT && CPLX) ? 2 : 1;   // column groups per (matrix, half)
  static constexpr int TN = 256 / NCG;                // output columns of a tile
  static constexpr int ACC = (CPLX ? 2 : 1) * TN;     // tensor-memory columns of one accumulator
  static constexpr int NBUF = 512 / ACC >= 2 ? 2 : 1;
  static constexpr int TMEM_COLS = 512;
  static constexpr int KSTEPS = ROT ? 2 * (TC_BJ_NB / 2) / NCG : 256 / KS;  // stages per tile
  static constexpr int EPI_WARPS = 8;
  static constexpr int CVT_WARPS = RAW ? 4 : 0;
  static constexpr int THREADS = 32 * (2 + EPI_WARPS + CVT_WARPS);
  static constexpr int XSTAGE = EPI_WARPS * 32 * 17 * 4;  // epilogue transpose staging, 32 x 16 per warp
  // one CTA per SM: it holds all 512 tensor-memory columns
  static constexpr size_t SMEM_USED = (size_t)STAGES * STAGE_BYTES + 1024 + 256 + XSTAGE;
  static constexpr size_t SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
};

constexpr int kMaxThreads = 448;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue, (RAW) 10-13 converters
constexpr int kPlane = 256 * 256;

struct TcParams {
  long batch;
  int conj_x, conj_y;
  int round;     // ROT: the block-Jacobi round whose pairs R rotates
  int conj_out;  // conjugate the result before it is written
  int withhold;  // failure-detection test: issue no loads, so every wait runs out
  int plain_n, plain_t;  // write out_n / out_t as plain float32 planes (no hi / lo split)
  float alpha, beta;
  float* out_n;
  float* out_t;
  int* err;
};

// Pair k of round r of the circle ordering of the TC_BJ_NB column blocks (p < q), as rr_pair.
__device__ __forceinline__ void block_pair(int r, int k, int& p, int& q) {
  constexpr int n = TC_BJ_NB;
  int a, b;
  if (k == 0) {
    a = n - 1;
    b = r;
  } else {
    a = (r + k) % (n - 1);
    b = (r - k + n - 1) % (n - 1);
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Output column block of accumulator slot `slot` (16 columns) of column group cg.  Full product:
// the slots are the blocks in order.  ROT: slot 2 j + w of group cg is block p (w = 0) or q (w =
// 1) of pair cg * (pairs per group) + j.
template <bool ROT, int NCG>
__device__ __forceinline__ int slot_block(int round, int cg, int slot) {
  if constexpr (!ROT) {
    return slot;
  } else {
    int bp, bq;
    block_pair(round, cg * (TC_BJ_NB / 2 / NCG) + (slot >> 1), bp, bq);
    return (slot & 1) ? bq : bp;
  }
}

template <bool CPLX, bool ROT>
__global__ void __launch_bounds__(kMaxThreads, 1)
    k_tcgemm(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my, const TcParams p) {
  using C = TcCfg<CPLX, ROT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* cvt = empty + C::STAGES;    // RAW: the stage's x is split
  uint64_t* tfull = cvt + C::STAGES;    // [NBUF]
  uint64_t* tempty = tfull + 2;         // [NBUF]
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  float* xst = reinterpret_cast<float*>(base + C::STAGES * C::STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long ntiles = 2L * C::NCG * p.batch;
  // tile t: matrix t / (2 NCG), row half (t / NCG) & 1, column group t % NCG
  auto tile = [&](long t, int& b, int& h, int& cg) {
    b = (int)(t / (2 * C::NCG));
    h = (int)((t / C::NCG) & 1);
    cg = (int)(t % C::NCG);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&cvt[s], C::CVT_WARPS > 0 ? C::CVT_WARPS : 1);
    }
    for (int i = 0; i < C::NBUF; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], C::EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_barrier_init();
    prefetch_tensormap(&mx);
    prefetch_tensormap(&my);
  }
  if (warp == 1) {
    tmem_alloc(tslot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued = 0, iph = 0;  // per stage: a load was issued, and the phase it completes
      for (long t = blockIdx.x; t < ntiles && !*abort && !p.withhold; t += gridDim.x) {
        int b, h, cg;
        tile(t, b, h, cg);
        for (int kb = 0; kb < C::KSTEPS; ++kb) {
          if (!mbar_wait(&empty[s], ph ^ 1, abort)) break;
          issued |= 1u << s;
          iph = (iph & ~(1u << s)) | (ph << s);
          mbar_arrive_expect_tx(&full[s], C::TX_BYTES);
          unsigned char* st = base + s * C::STAGE_BYTES;
          // K slice of this stage; ROT: stage kb is block (kb & 1 ? q : p) of the group's pair kb / 2
          static_assert(!ROT || TC_BJ_BS == C::KS, "a rotation stage spans one block");
          int kslice = kb, bp = 0, bq = 0;
          if constexpr (ROT) {
            block_pair(p.round, cg * (TC_BJ_NB / 2 / C::NCG) + (kb >> 1), bp, bq);
            kslice = (kb & 1) ? bq : bp;
          }
          if constexpr (C::RAW) {
            for (int pl = 0; pl < C::NPX; ++pl)
              tma_load_4d(st + C::RAWOFF + pl * C::XB, &mx, &full[s], 0, 128 * h, kslice * (C::KS / 4),
                          b * C::NPX + pl);
          }
          for (int pl = 0; pl < C::NPL; ++pl) {
            if constexpr (!C::RAW)
              tma_load_4d(st + pl * C::XB, &mx, &full[s], 0, 128 * h, kslice * (C::KS / 4), b * C::NPL + pl);
            if constexpr (ROT) {
              // the pair's compact 32 x 32 block: its 32 rows, the K half of this stage's block
              const int jg = cg * (TC_BJ_NB / 2 / C::NCG) + (kb >> 1);
              tma_load_4d(st + C::NPL * C::XB + pl * C::YB, &my, &full[s], 0, 2 * TC_BJ_BS * jg,
                          (kb & 1) * (C::KS / 4), b * C::NPL + pl);
            } else {
              tma_load_4d(st + C::NPL * C::XB + pl * C::YB, &my, &full[s], 0, 0, kslice * (C::KS / 4),
                          b * C::NPL + pl);
            }
          }
          if (++s == C::STAGES) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      if (*abort) {
        // copies still in flight land before the CTA leaves: wait (bounded) for the phase each
        // issued stage completes; a completed one returns at once
        volatile int never = 0;
        for (int k = 0; k < C::STAGES; ++k)
          if (issued & (1u << k)) mbar_wait(&full[k], (iph >> k) & 1u, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t XLBO = 128 * 16, YLBO = C::YR * 16, SBO = 128;
      // products of one K step: (x plane, y plane, accumulator column, negate)
      // real: hi hi, hi lo, lo hi.  Complex x = xr + i sx xi, y = yr + i sy yi (s = -1 when
      // conjugated): Dr = xr yr^T - sx sy xi yi^T, Di = sy xr yi^T + sx xi yr^T.
      const int sx = p.conj_x ? -1 : 1, sy = p.conj_y ? -1 : 1;
      int s = 0;
      uint32_t ph = 0;
      int local = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++local) {
        const int bi = local % C::NBUF;
        const uint32_t use = (uint32_t)(local / C::NBUF);  // earlier uses of this accumulator
        if (!mbar_wait(&tempty[bi], (use & 1) ^ 1, abort)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(bi * C::ACC);
        bool ok = true;
        for (int kb = 0; kb < C::KSTEPS; ++kb) {
          if (!mbar_wait(&full[s], ph, abort) || (C::RAW && !mbar_wait(&cvt[s], ph, abort))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + s * C::STAGE_BYTES);
          const uint32_t xs = st, ys0 = st + C::NPL * C::XB;
          // ROT: the stage's K slice feeds the accumulator slots of both blocks of its pair (N =
          // 2 TC_BJ_BS, adjacent slots), accumulated only over the pair's 2 stages (R is zero
          // elsewhere)
#pragma unroll
          for (int cb = 0; cb < C::NYS; ++cb) {
            const uint32_t ys = ys0 + cb * C::NPL * C::YB;
            const uint32_t c0 = ROT ? (uint32_t)TC_BJ_BS * (uint32_t)(2 * (kb >> 1)) : 0u;
            constexpr int NN = ROT ? 2 * TC_BJ_BS : 256;
#pragma unroll
            for (int ks = 0; ks < C::KS / 8; ++ks) {
              auto mma = [&](int xp, int yp, uint32_t col, int neg, bool first) {
                const uint64_t ad = smem_desc(xs + xp * C::XB + ks * 2 * XLBO, XLBO, SBO);
                const uint64_t bd = smem_desc(ys + yp * C::YB + ks * 2 * YLBO, YLBO, SBO);
                mma_tf32(acc + c0 + col, ad, bd, idesc_tf32(128, NN, neg, 0), first ? 0u : 1u);
              };
              const bool f0 = (ROT ? (kb & 1) == 0 : kb == 0) && ks == 0;
              if constexpr (!CPLX) {
                mma(0, 0, 0, 0, f0);
                mma(0, 1, 0, 0, false);
                mma(1, 0, 0, 0, false);
              } else {
                const int nr = (sx * sy > 0) ? 1 : 0;  // Dr: - sx sy xi yi^T
                mma(0, 0, 0, 0, f0);
                mma(0, 1, 0, 0, false);
                mma(1, 0, 0, 0, false);
                mma(2, 2, 0, nr, false);
                mma(2, 3, 0, nr, false);
                mma(3, 2, 0, nr, false);
                const int ni1 = sy < 0 ? 1 : 0, ni2 = sx < 0 ? 1 : 0;
                mma(0, 2, C::TN, ni1, f0);
                mma(0, 3, C::TN, ni1, false);
                mma(1, 2, C::TN, ni1, false);
                mma(2, 0, C::TN, ni2, false);
                mma(2, 1, C::TN, ni2, false);
                mma(3, 0, C::TN, ni2, false);
              }
            }
          }
          mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
          if (++s == C::STAGES) {
            s = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(&tfull[bi]);
      }
      if (*abort) {
        // every MMA issued so far completes before this commit's arrival
        mma_commit(drain);
        volatile int never = 0;
        mbar_wait(drain, 0, &never);
      }
    }
  } else if (warp >= 2 + C::EPI_WARPS) {
    // ---- (RAW) converters: split each landed K slice of x into hi / lo planes
    if constexpr (C::RAW) {
      const int ct = threadIdx.x - 32 * (2 + C::EPI_WARPS);  // 0 .. 127
      constexpr int Q4 = C::XB / 16;                         // float4 per plane slice
      int s = 0;
      uint32_t ph = 0;
      bool go = true;
      for (long t = blockIdx.x; go && t < ntiles; t += gridDim.x) {
        for (int kb = 0; kb < C::KSTEPS; ++kb) {
          // warp-uniform: every lane of the warp takes the same exit
          const bool ok = !*abort && mbar_wait(&full[s], ph, abort);
          if (!__all_sync(0xffffffffu, ok)) {
            go = false;
            break;
          }
          unsigned char* st = base + s * C::STAGE_BYTES;
          const float4* raw = reinterpret_cast<const float4*>(st + C::RAWOFF);
          float4* spl = reinterpret_cast<float4*>(st);
          for (int i = ct; i < C::NPX * Q4; i += 32 * C::CVT_WARPS) {
            const int pl = i / Q4, o = i - pl * Q4;
            const float4 v = raw[i];
            float4 hi;
            hi.x = tf32_hi(v.x);
            hi.y = tf32_hi(v.y);
            hi.z = tf32_hi(v.z);
            hi.w = tf32_hi(v.w);
            spl[(2 * pl) * Q4 + o] = hi;
            spl[(2 * pl + 1) * Q4 + o] = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&cvt[s]);
          if (++s == C::STAGES) {
            s = 0;
            ph ^= 1;
          }
        }
      }
    }
  } else {
    // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) ... + 31, i.e. output rows, and
    // the accumulator slots of its parity (w - 2) / 4
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int m = 32 * q + lane;
    float* tile_st = xst + (warp - 2) * (32 * 17);
    int local = 0;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
      int b, h, cg;
      tile(t, b, h, cg);
      const int bi = local % C::NBUF;
      const uint32_t use = (uint32_t)(local / C::NBUF);
      // warp-uniform decision: the tensor-memory loads below are .sync.aligned
      const bool ok = !*abort && mbar_wait(&tfull[bi], use & 1, abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t acc = tmem + (uint32_t)(bi * C::ACC) + ((uint32_t)(32 * q) << 16);
      const int gr = 128 * h + m;  // output row
      float* on = p.out_n ? p.out_n + (size_t)b * (p.plain_n ? C::NPX : C::NPL) * kPlane : nullptr;
      float* ot = p.out_t ? p.out_t + (size_t)b * (p.plain_t ? C::NPX : C::NPL) * kPlane : nullptr;
      for (int slot = half; slot < C::TN / 16; slot += 2) {
        const int n0 = 16 * slot_block<ROT, C::NCG>(p.round, cg, slot);  // output column
        float vr[16], vi[16];
        tmem_ld16(acc + 16 * slot, vr);
        if constexpr (CPLX) tmem_ld16(acc + C::TN + 16 * slot, vi);
        const float ci = p.conj_out ? -p.alpha : p.alpha;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          vr[j] = p.alpha * vr[j] + ((gr == n0 + j) ? p.beta : 0.f);
          if constexpr (CPLX) vi[j] = ci * vi[j];
        }
        if (on && p.plain_n) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int off = ((n0 / 4 + c) * 256 + gr) * 4;
            *reinterpret_cast<float4*>(on + off) = make_float4(vr[4 * c], vr[4 * c + 1], vr[4 * c + 2], vr[4 * c + 3]);
            if constexpr (CPLX)
              *reinterpret_cast<float4*>(on + kPlane + off) =
                  make_float4(vi[4 * c], vi[4 * c + 1], vi[4 * c + 2], vi[4 * c + 3]);
          }
        } else if (on) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int off = ((n0 / 4 + c) * 256 + gr) * 4;
            float4 hi, lo;
            hi.x = tf32_hi(vr[4 * c]);
            hi.y = tf32_hi(vr[4 * c + 1]);
            hi.z = tf32_hi(vr[4 * c + 2]);
            hi.w = tf32_hi(vr[4 * c + 3]);
            lo.x = vr[4 * c] - hi.x;
            lo.y = vr[4 * c + 1] - hi.y;
            lo.z = vr[4 * c + 2] - hi.z;
            lo.w = vr[4 * c + 3] - hi.w;
            *reinterpret_cast<float4*>(on + off) = hi;
            *reinterpret_cast<float4*>(on + kPlane + off) = lo;
            if constexpr (CPLX) {
              hi.x = tf32_hi(vi[4 * c]);
              hi.y = tf32_hi(vi[4 * c + 1]);
              hi.z = tf32_hi(vi[4 * c + 2]);
              hi.w = tf32_hi(vi[4 * c + 3]);
              lo.x = vi[4 * c] - hi.x;
              lo.y = vi[4 * c + 1] - hi.y;
              lo.z = vi[4 * c + 2] - hi.z;
              lo.w = vi[4 * c + 3] - hi.w;
              *reinterpret_cast<float4*>(on + 2 * kPlane + off) = hi;
              *reinterpret_cast<float4*>(on + 3 * kPlane + off) = lo;
            }
          }
        }
        if (ot) {
          // D^T through a per-warp shared-memory tile: the warp holds rows gr0 .. gr0 + 31 and
          // columns n0 .. n0 + 15; in D^T's KC4 layout a 4-row chunk of one column is one float4,
          // and the 16 columns of a chunk are 256 contiguous bytes, so each half-warp stores one
          // chunk row in one contiguous segment.
          // plain: parts re (, im); split: parts re hi, re lo (, im hi, im lo)
          const int gr0 = 128 * h + 32 * q;
          const int nparts = p.plain_t ? C::NPX : C::NPL;
#pragma unroll
          for (int part = 0; part < C::NPL; ++part) {
            if (part >= nparts) break;
            const bool im = p.plain_t ? part == 1 : part >= 2;
            const float* v = im ? vi : vr;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float hv = tf32_hi(v[j]);
              tile_st[lane * 17 + j] = p.plain_t ? v[j] : ((part & 1) ? v[j] - hv : hv);
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int qq = lane + 32 * i, c = qq >> 4, n = qq & 15;
              const float4 w4 = make_float4(tile_st[(4 * c) * 17 + n], tile_st[(4 * c + 1) * 17 + n],
                                            tile_st[(4 * c + 2) * 17 + n], tile_st[(4 * c + 3) * 17 + n]);
              *reinterpret_cast<float4*>(ot + part * kPlane + ((gr0 / 4 + c) * 256 + n0 + n) * 4) = w4;
            }
            __syncwarp();
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[bi]);
    }
  }

  // ---- exit (the producer and the MMA thread have drained their work after an abort)
  __syncthreads();
  if (threadIdx.x == 0 && *abort && p.err) atomicExch(p.err, 1);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// Tensor map over `planes` KC4 planes of 256 rows x kdim columns at `ptr`: dims (k % 4, r, k / 4,
// plane), box (4, rows, 4, 1).  kdim = 256 for the matrices, 32 for the compact rotations.
bool make_map(CUtensorMap* map, const float* ptr, long planes, int rows, int kdim = 256) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[4] = {4, 256, (cuuint64_t)(kdim / 4), (cuuint64_t)planes};
  cuuint64_t strides[3] = {16, 256 * 16, (cuuint64_t)256 * kdim * 4};
  cuuint32_t box[4] = {4, (cuuint32_t)rows, 4, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

template <bool CPLX, bool ROT>
cudaError_t launch(const TcGemm& g, cudaStream_t s) {
  using C = TcCfg<CPLX, ROT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tcgemm<CPLX, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  CUtensorMap mx, my;
  if (!make_map(&mx, g.x, g.batch * (C::RAW ? C::NPX : C::NPL), 128) ||
      !make_map(&my, g.y, g.batch * C::NPL, C::YR, ROT ? 2 * TC_BJ_BS : 256))
    return cudaErrorInvalidValue;
  TcParams p;
  p.batch = g.batch;
  p.conj_x = g.conj_x;
  p.conj_y = g.conj_y;
  p.round = g.round;
  p.conj_out = g.conj_out;
  p.withhold = g.withhold_loads;
  p.plain_n = g.plain_n;
  p.plain_t = g.plain_t;
  p.alpha = g.alpha;
  p.beta = g.beta;
  p.out_n = g.out_n;
  p.out_t = g.out_t;
  p.err = g.err;
  const long tiles = 2L * C::NCG * g.batch;
  const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
  k_tcgemm<CPLX, ROT><<<grid, C::THREADS, C::SMEM, s>>>(mx, my, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_gemm256(const TcGemm& g, cudaStream_t s) {
  if (g.batch <= 0) return cudaSuccess;
  if (!g.x || !g.y || (!g.out_n && !g.out_t)) return cudaErrorInvalidValue;
  if (((uintptr_t)g.x | (uintptr_t)g.y | (uintptr_t)g.out_n | (uintptr_t)g.out_t) & 15)
    return cudaErrorInvalidValue;
  return g.cplx ? launch<true, false>(g, s) : launch<false, false>(g, s);
}

cudaError_t tc_rot256(const TcGemm& g, cudaStream_t s) {
  if (g.batch <= 0) return cudaSuccess;
  if (!g.x || !g.y || (!g.out_n && !g.out_t) || g.round < 0 || g.round > TC_BJ_NB - 2)
    return cudaErrorInvalidValue;
  if (((uintptr_t)g.x | (uintptr_t)g.y | (uintptr_t)g.out_n | (uintptr_t)g.out_t) & 15)
    return cudaErrorInvalidValue;
  return g.cplx ? launch<true, true>(g, s) : launch<false, true>(g, s);
}

}  // namespace ve

// ---------------------------------------------------------------- failure-detection self-test
extern "C" int ve_selftest_bounded_wait(double* seconds) {
  using namespace ve;
  if (!seconds) return VE_EINVAL;
  cudaGetLastError();
  const size_t mat = (size_t)2 * kPlane * sizeof(float);  // one real split matrix
  float* buf = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&buf, 3 * mat) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (buf) cudaFree(buf);
    return VE_ENOMEM;
  }
  int rc = VE_OK;
  int h_err = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TcGemm g;
  g.x = buf;
  g.y = buf + 2 * kPlane;
  g.out_n = buf + 4 * kPlane;
  g.batch = 1;
  g.err = err;
  float ms = 0.f;
  bool ok = cudaMemset(buf, 0, 3 * mat) == cudaSuccess && cudaMemset(err, 0, sizeof(int)) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  // 1. loads withheld: the waits must run out, the kernel report it and return
  g.withhold_loads = 1;
  ok = ok && cudaEventRecord(e0, 0) == cudaSuccess && tc_gemm256(g, 0) == cudaSuccess &&
       cudaEventRecord(e1, 0) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
       cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
       cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  if (!ok) rc = VE_ECUDA;
  else if (h_err != 1) rc = VE_ETIMEOUT;  // the stall went unreported
  // 2. the context is still usable: the same product with its loads runs clean
  if (rc == VE_OK) {
    g.withhold_loads = 0;
    h_err = 0;
    ok = cudaMemset(err, 0, sizeof(int)) == cudaSuccess && tc_gemm256(g, 0) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess &&
         cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) rc = VE_ECUDA;
    else if (h_err != 0) rc = VE_ETIMEOUT;
  }
  *seconds = ms * 1e-3;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(err);
  return rc;
}
