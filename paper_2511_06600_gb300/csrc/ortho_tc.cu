// Tensor-core Gram matrix for the FP32 form of CholQR2 (Algorithm 1 step 4):
// G_aug = [V 1]^T [V 1] on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators).  FP32 accuracy from TF32 inputs by the 3-product split
// x = hi + lo (hi = tf32(x), lo = x - hi): x y ~ hi hi' + hi lo' + lo hi'.
// The all-ones column gives the column sums (and n) for free.
//
// One CTA per SM-sized chunk of rows.  Per 32-row slab the CTA writes the
// transposed slab (basis index x 32 rows, K-major, 128-byte swizzle) as hi and
// lo tiles into shared memory (double-buffered), and one thread issues the
// MMAs of the upper block rows: block b covers basis rows [128b, 128b+128)
// against basis columns [128b, Kq).  Completion is tracked by tcgen05.commit
// on an mbarrier per stage; every wait is bounded and a timeout sets *err.
// The epilogue moves the FP32 accumulators from TMEM to per-CTA FP32 partials
// (no FP64 work on the SM); k_gram_tc_reduce widens them and sums in FP64.
//
// A basis stored in BF16 (BF = true) enters the same MMAs: a BF16 value is
// exact in TF32 (8 significant bits within TF32's 11), so its lo part is
// zero and one product hi hi' gives the exact products of the stored
// values, accumulated in FP32 — what a BF16-input MMA with FP32 accumulation
// computes.  The apply likewise needs hi(V) hi(R^-1) + hi(V) lo(R^-1), and
// rounds Q to BF16 on the store.
#include <cuda_bf16.h>

#include "internal.h"
#include "umma.cuh"

namespace hef {

namespace {

using namespace umma;

constexpr int kApThreads = 512;  // apply: 16 warps load and split the A tiles
constexpr int kGrThreads = 512;  // Gram: 16 warps load and split the slabs
constexpr int kSlab = 32;                    // V rows per stage (128 B of fp32)
constexpr uint32_t kWaitIters = 1u << 20;    // bounded mbarrier waits

struct GramTcArgs {
  const float* V;
  const __nv_bfloat16* Vb;  // BF16 basis (the BF form of the kernels)
  long long ldv;
  int n, K, Kq, nb;
  int rows_per_cta;
  int gmask[4];  // block rows of G_aug computed by CTA group blockIdx.y (bit b: rows 128b..)
  float* part;   // gridDim.x x Kq x Kq FP32 partials (the accumulators as they are)
  int* err;
};

// Slab loader: thread tid owns the float4 slots f = tid + 256 k of a slab
// (slab row f % 32, basis columns 4 (f / 32) .. + 3); values past K are the
// ones column (index K) or zero, rows past the chunk are zero.
template <bool BF>
__device__ __forceinline__ float gram_elem(const GramTcArgs& a, long long row, int c) {
  if constexpr (BF) return __bfloat162float(a.Vb[row * a.ldv + c]);
  else return a.V[row * a.ldv + c];
}

template <int PER, bool BF>
__device__ __forceinline__ void gram_load_slab(const GramTcArgs& a, long long rowbase, long long r1,
                                               float4 (&buf)[PER]) {
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int f = threadIdx.x + kGrThreads * k;
    const int r = f & (kSlab - 1), c0 = 4 * (f >> 5);
    if (c0 >= a.Kq) continue;  // padding rows of the tile: zero, written once
    const long long row = rowbase + r;
    const bool valid = row < r1;
    if (valid && c0 + 3 < a.K) {
      if constexpr (BF) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(a.Vb + row * a.ldv + c0));
        const __nv_bfloat162 h0 = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
        const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
        const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
        buf[k] = make_float4(f0.x, f0.y, f1.x, f1.y);
      } else {
        buf[k] = __ldg(reinterpret_cast<const float4*>(a.V + row * a.ldv + c0));
      }
    } else {
      float x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u;
        x[u] = !valid ? 0.f : (c < a.K ? gram_elem<BF>(a, row, c) : (c == a.K ? 1.f : 0.f));
      }
      buf[k] = make_float4(x[0], x[1], x[2], x[3]);
    }
  }
}

// G_aug block rows of this CTA's group: block b covers basis rows
// [128b, 128b+128) against basis columns [128b, Kq) (N_b = Kq - 128b, issued
// as MMAs of N <= 256); its accumulator occupies TMEM columns from the sum of
// the earlier blocks' N in the group.  NB blocks of 128 rows pad the
// transposed slab; STAGES shared-memory stages (2, or 1 when two do not fit).
template <int NB, int STAGES, bool BF>
__global__ void __launch_bounds__(kGrThreads, 1) k_gram_tc(GramTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int Mpad = NB * 128;
  constexpr int PER = kSlab * (Mpad / 4) / kGrThreads;  // float4 slots per thread
  const uint32_t tile_bytes = (uint32_t)Mpad * 128u;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGES * tile_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gmask = a.gmask[blockIdx.y];
  int toff[NB];  // TMEM column of each block of the group
  int used = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    toff[b] = used;
    if ((gmask >> b) & 1) used += a.Kq - 128 * b;
  }
  uint32_t ncols = 32;
  while (ncols < (uint32_t)used) ncols <<= 1;

  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < STAGES; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // basis rows [Kq, Mpad) of the transposed tiles are zero for every slab
  for (int q = 0; q < 2 * STAGES; ++q) {
    unsigned char* tile = base + (size_t)q * tile_bytes;
    for (int e = tid; e < (Mpad - a.Kq) * 32; e += kGrThreads)
      *reinterpret_cast<float*>(tile + sw128_offset(a.Kq + e / 32, e % 32)) = 0.f;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const long long r0 = (long long)blockIdx.x * a.rows_per_cta;
  const long long r1 = min((long long)a.n, r0 + a.rows_per_cta);
  const int nslab = r1 > r0 ? (int)((r1 - r0 + kSlab - 1) / kSlab) : 0;
  bool ok = true;
  int committed = 0;  // slabs whose MMAs were issued
  float4 cur[PER], nxt[PER];
  if (nslab > 0) gram_load_slab<PER, BF>(a, r0, r1, cur);

  for (int t = 0; t < nslab; ++t) {
    const int s = t % STAGES;
    // next slab's loads are in flight while this one is converted and issued
    if (t + 1 < nslab) gram_load_slab<PER, BF>(a, r0 + (long long)(t + 1) * kSlab, r1, nxt);
    if (t >= STAGES) ok = ok && mbar_wait(&bars[s], ((t - STAGES) / STAGES) & 1, kWaitIters);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    unsigned char* hi = base + (size_t)s * 2 * tile_bytes;
    unsigned char* lo = hi + tile_bytes;
    // transposed slab: element (basis i, slab row r) at sw128_offset(i, r)
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int f = tid + kGrThreads * k;
      const int r = f & (kSlab - 1), c0 = 4 * (f >> 5);
      if (c0 >= a.Kq) continue;  // warp-uniform
      const float x[4] = {cur[k].x, cur[k].y, cur[k].z, cur[k].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t off = sw128_offset(c0 + u, r);
        if constexpr (BF) {
          *reinterpret_cast<float*>(hi + off) = x[u];  // exact in TF32; lo = 0
        } else {
          const float h = tf32_round(x[u]);
          *reinterpret_cast<float*>(hi + off) = h;
          *reinterpret_cast<float*>(lo + off) = x[u] - h;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) cur[k] = nxt[k];
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t shi = smem_u32(hi), slo = smem_u32(lo);
#pragma unroll
      for (int ks = 0; ks < kSlab / 8; ++ks) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (!((gmask >> b) & 1)) continue;
          const int Nb = a.Kq - 128 * b;
          const uint32_t aoff = (uint32_t)b * 128u * 128u + (uint32_t)ks * 32u;
          const uint32_t acc = (t > 0 || ks > 0) ? 1u : 0u;
          for (int h0 = 0; h0 < Nb; h0 += 256) {
            const int Nh = min(256, Nb - h0);
            const uint32_t boff = aoff + (uint32_t)h0 * 128u;
            const uint32_t d = tmem + (uint32_t)(toff[b] + h0);
            const uint32_t id = idesc_tf32(128, Nh);
            mma_tf32(d, desc_k_sw128(shi + aoff), desc_k_sw128(shi + boff), id, acc);
            if constexpr (!BF) {
              mma_tf32(d, desc_k_sw128(shi + aoff), desc_k_sw128(slo + boff), id, 1u);
              mma_tf32(d, desc_k_sw128(slo + aoff), desc_k_sw128(shi + boff), id, 1u);
            }
          }
        }
      }
      mma_commit(&bars[s]);
    }
    committed = t + 1;
  }
  // the last commit covers every MMA issued before it
  if (committed > 0) {
    const int t = committed - 1;
    const bool done = mbar_wait(&bars[t % STAGES], (t / STAGES) & 1, kWaitIters);
    ok = ok && done;
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();
  float* P = a.part + (size_t)blockIdx.x * a.Kq * a.Kq;
  if (ok && committed > 0) {
    // warp w reads TMEM lanes 32 (w mod 4) ..; the kGrThreads / 128 warps of a
    // lane quarter take every (kGrThreads / 128)-th group of 8 columns
    const int q = warp & 3, part = warp >> 2;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!((gmask >> b) & 1)) continue;
      const int ncol = a.Kq - 128 * b;
      const int i = b * 128 + q * 32 + lane;
      for (int c8 = part; c8 < ncol / 8; c8 += kGrThreads / 128) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)toff[b] + (uint32_t)c8 * 8u, v);
        tmem_wait_ld();
        const int j0 = b * 128 + c8 * 8;
        if (i < a.Kq && j0 + 7 >= i) {  // upper triangle only (the reducer reads i <= j)
#pragma unroll
          for (int u = 0; u < 8; ++u) P[(size_t)i * a.Kq + j0 + u] = v[u];
        }
      }
    }
  } else {
    // zero this group's block rows
    for (int e = tid; e < a.Kq * a.Kq; e += kGrThreads)
      if ((gmask >> ((e / a.Kq) / 128)) & 1) P[e] = 0.f;
    if (!ok && tid == 0) atomicExch(a.err, 1);
    if (!ok && committed > 0) {  // let MMAs in flight finish before TMEM is released
      const int t = committed - 1;
      mbar_wait(&bars[t % STAGES], (t / STAGES) & 1, kWaitIters);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// G (K x K, FP64) and c (K): fixed-order FP64 sums of the per-CTA FP32
// partials of G_aug (column K holds the column sums).  Eight lanes per entry:
// lane l of the eight sums partials l, l + 8, ... in order, then a fixed
// shuffle tree; a warp takes four consecutive entries per round.
__global__ void k_gram_tc_reduce(const float* __restrict__ part, int K, int Kq, int nchunk,
                                 double* G, double* c) {
  const long long KK = (long long)K * K, total = KK + K;
  const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const size_t stride = (size_t)Kq * Kq;
  for (long long wb = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; wb < total;
       wb += nwarps * 4) {
    const long long idx = wb + grp;
    int i = 0, j = 0;
    bool act = idx < total;
    if (act) {
      if (idx < KK) {
        i = (int)(idx / K), j = (int)(idx % K);
        act = i <= j;
      } else {
        i = (int)(idx - KK), j = K;
      }
    }
    double s = 0.0;
    if (act) {
      const float* p = part + (size_t)i * Kq + j;
      int q = sub;
      for (; q + 24 < nchunk; q += 32) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcg(p + (size_t)(q + 8 * u) * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) s += (double)v[u];
      }
      for (; q < nchunk; q += 8) s += (double)__ldcg(p + (size_t)q * stride);
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (act && sub == 0) {
      if (j < K) {
        G[(size_t)i * K + j] = s;
        G[(size_t)j * K + i] = s;
      } else {
        c[i] = s;
      }
    }
  }
}

// ---------------------------------------------------------------- apply

// B operand and mean correction of the apply: RinvT_hi/lo[j][i] (Kq x Kd,
// row-major) = hi/lo split of Rinv[i][j]; muR[j] = sum_i mu_i Rinv[i][j].
__global__ void k_rinv_split(const float* __restrict__ Rinv, const float* __restrict__ mu, int K,
                             int Kp, int Kq, int Kd, float* RtH, float* RtL, float* muR) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)Kq * Kd;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / Kd), i = (int)(idx % Kd);
    const float x = (i < K && j < K) ? Rinv[(size_t)i * Kp + j] : 0.f;
    const float h = tf32_round(x);
    RtH[idx] = h;
    RtL[idx] = x - h;
  }
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < Kq;
       j += (long long)gridDim.x * blockDim.x) {
    float s0 = 0.f, s1 = 0.f;
    if (j < K) {
      int i = 0;
      for (; i + 1 <= (int)j; i += 2) {
        s0 += mu[i] * Rinv[(size_t)i * Kp + j];
        s1 += mu[i + 1] * Rinv[(size_t)(i + 1) * Kp + j];
      }
      if (i <= (int)j) s0 += mu[i] * Rinv[(size_t)i * Kp + j];
    }
    muR[j] = s0 + s1;
  }
}

struct ApplyTcArgs {
  float* V;
  __nv_bfloat16* Vb;  // BF16 basis (the BF form), Q rounded to BF16
  long long ldv;
  int n, K, Kq, Kd;
  const float* RtH;
  const float* RtL;
  const float* muR;
  int* err;
};

// Q = (V - 1 mu^T) Rinv = V Rinv - 1 (mu^T Rinv), in place, 128-row tiles.
// K block ka covers basis values [32 ka, 32 ka + 32): its A tile holds those
// values of the tile's rows (hi and lo), its B tile the rows j >= 32 ka of
// Rinv^T (Rinv is upper triangular, so block ka feeds output columns
// j >= 32 ka only).  RESB: every B tile stays resident in shared memory
// (staged once per CTA); otherwise B is staged with A for every block.
template <bool RESB, int STAGES, bool BF>
__global__ void __launch_bounds__(kApThreads, 1) k_apply_tc(ApplyTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nka = a.Kd / 32;
  const uint32_t a_bytes = 128u * 128u;  // one A tile (hi or lo)
  // B region: tile ka (hi, then lo) at boff(ka); rows Kq - 32 ka
  auto brows = [&](int ka) { return a.Kq - 32 * ka; };
  auto boff = [&](int ka) {  // bytes before B tile pair ka
    return RESB ? (uint32_t)(ka * a.Kq - 16 * ka * (ka - 1)) * 256u : 0u;
  };
  const uint32_t b_region = RESB ? boff(nka) : 2u * (uint32_t)a.Kq * 128u;
  const uint32_t stage_bytes = 2 * a_bytes + (RESB ? 0u : b_region);
  unsigned char* bbase = base;
  unsigned char* sbase = base + (RESB ? b_region : 0u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + STAGES * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)a.Kq) ncols <<= 1;
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < STAGES; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B tile ka: row jr = Rinv^T row 32 ka + jr, basis values [32 ka, 32 ka + 32)
  auto stage_b = [&](int ka, unsigned char* bhi, unsigned char* blo) {
    const int c0 = ka * 32, nr = brows(ka);
    for (int f = tid; f < nr * 8; f += kApThreads) {
      const int jr = f >> 3, q = f & 7;
      const size_t src = (size_t)(c0 + jr) * a.Kd + c0 + 4 * q;
      const uint32_t off = sw128_offset(jr, 4 * q);
      *reinterpret_cast<float4*>(bhi + off) = __ldg(reinterpret_cast<const float4*>(a.RtH + src));
      *reinterpret_cast<float4*>(blo + off) = __ldg(reinterpret_cast<const float4*>(a.RtL + src));
    }
  };
  if (RESB) {
    for (int ka = 0; ka < nka; ++ka) {
      unsigned char* bhi = bbase + boff(ka);
      stage_b(ka, bhi, bhi + (uint32_t)brows(ka) * 128u);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = (a.n + 127) / 128;
  bool ok = true;
  uint32_t uses0 = 0u, uses1 = 0u;  // commits per stage so far
  int g = 0;                        // global stage counter (alternates buffers)
  int last_stage = -1;
  // A slots of a stage: f = tid + kApThreads k -> tile row f / 8, basis
  // values 32 ka + 4 (f % 8) .. + 3; the next stage's are loaded while this
  // one is used
  constexpr int kAPer = 128 * 8 / kApThreads;
  auto load_a = [&](int tile, int ka, float4 (&buf)[kAPer]) {
#pragma unroll
    for (int k = 0; k < kAPer; ++k) {
      const int f = tid + kApThreads * k;
      const int r = f >> 3, q = f & 7;
      const long long row = (long long)tile * 128 + r;
      const int col = ka * 32 + 4 * q;
      if (tile < ntiles && row < a.n && col + 3 < a.K) {
        if constexpr (BF) {
          const uint2 u = __ldg(reinterpret_cast<const uint2*>(a.Vb + row * a.ldv + col));
          const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
          const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
          buf[k] = make_float4(f0.x, f0.y, f1.x, f1.y);
        } else {
          buf[k] = __ldg(reinterpret_cast<const float4*>(a.V + row * a.ldv + col));
        }
      } else {
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = tile < ntiles && row < a.n && col + u < a.K;
          if constexpr (BF) x[u] = in ? __bfloat162float(a.Vb[row * a.ldv + col + u]) : 0.f;
          else x[u] = in ? a.V[row * a.ldv + col + u] : 0.f;
        }
        buf[k] = make_float4(x[0], x[1], x[2], x[3]);
      }
    }
  };
  float4 cur[kAPer], nxt[kAPer];
  load_a(blockIdx.x, 0, cur);
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long row0 = (long long)tile * 128;
    for (int ka = 0; ka < nka; ++ka, ++g) {
      const int s = STAGES == 1 ? 0 : (g & 1);
      const uint32_t uses_s = s ? uses1 : uses0;
      if (ka + 1 < nka) load_a(tile, ka + 1, nxt);
      else load_a(tile + gridDim.x, 0, nxt);
      if (uses_s > 0) ok = ok && mbar_wait(&bars[s], (uses_s - 1) & 1, kWaitIters);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      unsigned char* ahi = sbase + (size_t)s * stage_bytes;
      unsigned char* alo = ahi + a_bytes;
      unsigned char* bhi;
      unsigned char* blo;
      if (RESB) {
        bhi = bbase + boff(ka);
        blo = bhi + (uint32_t)brows(ka) * 128u;
      } else {
        bhi = alo + a_bytes;
        blo = bhi + (uint32_t)a.Kq * 128u;
        stage_b(ka, bhi, blo);
      }
#pragma unroll
      for (int k = 0; k < kAPer; ++k) {
        const int f = tid + kApThreads * k;
        const int r = f >> 3, q = f & 7;
        const float x[4] = {cur[k].x, cur[k].y, cur[k].z, cur[k].w};
        const uint32_t off = sw128_offset(r, 4 * q);
        if constexpr (BF) {  // exact in TF32: no lo part
          *reinterpret_cast<float4*>(ahi + off) = make_float4(x[0], x[1], x[2], x[3]);
        } else {
          float h[4], l[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) h[u] = tf32_round(x[u]), l[u] = x[u] - h[u];
          *reinterpret_cast<float4*>(ahi + off) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(alo + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
      }
#pragma unroll
      for (int k = 0; k < kAPer; ++k) cur[k] = nxt[k];
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const int c0 = ka * 32;
        const int nr = brows(ka);
        const uint32_t sah = smem_u32(ahi), sal = smem_u32(alo);
        const uint32_t sbh = smem_u32(bhi), sbl = smem_u32(blo);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ko = (uint32_t)ks * 32u;
          // output columns c0 .. c0 + nr - 1, in MMAs of N <= 256
          for (int h0 = 0; h0 < nr; h0 += 256) {
            const int Nh = min(256, nr - h0);
            const uint32_t id = idesc_tf32(128, Nh);
            const uint32_t d = tmem + (uint32_t)(c0 + h0);
            const uint32_t bo = ko + (uint32_t)h0 * 128u;
            // block 0 covers every output column: its first K step starts them
            const uint32_t acc = (ka > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(d, desc_k_sw128(sah + ko), desc_k_sw128(sbh + bo), id, acc);
            mma_tf32(d, desc_k_sw128(sah + ko), desc_k_sw128(sbl + bo), id, 1u);
            if constexpr (!BF) mma_tf32(d, desc_k_sw128(sal + ko), desc_k_sw128(sbh + bo), id, 1u);
          }
        }
        mma_commit(&bars[s]);
      }
      if (s) ++uses1;
      else ++uses0;
      last_stage = s;
    }
    if (!ok) break;
    // tile done: wait for its last commit, then TMEM -> registers -> V
    {
      const uint32_t ul = last_stage ? uses1 : uses0;
      ok = ok && mbar_wait(&bars[last_stage], (ul - 1) & 1, kWaitIters);
    }
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    tc_fence_after();
    // warp w reads TMEM lanes 32 (w mod 4) ..; the kApThreads / 128 warps of
    // a lane quarter take every (kApThreads / 128)-th group of 8 columns
    const int q4 = warp & 3, part = warp >> 2;
    const long long row = row0 + q4 * 32 + lane;
    for (int c8 = part; c8 < a.Kq / 8; c8 += kApThreads / 128) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c8 * 8u, v);
      tmem_wait_ld();
      const int j0 = c8 * 8;
      if (BF && row < a.n) {
        if (j0 + 7 < a.K) {
          const float4 m0 = __ldg(reinterpret_cast<const float4*>(a.muR + j0));
          const float4 m1 = __ldg(reinterpret_cast<const float4*>(a.muR + j0 + 4));
          __nv_bfloat162 h[4];
          h[0] = __floats2bfloat162_rn(v[0] - m0.x, v[1] - m0.y);
          h[1] = __floats2bfloat162_rn(v[2] - m0.z, v[3] - m0.w);
          h[2] = __floats2bfloat162_rn(v[4] - m1.x, v[5] - m1.y);
          h[3] = __floats2bfloat162_rn(v[6] - m1.z, v[7] - m1.w);
          *reinterpret_cast<uint4*>(a.Vb + row * a.ldv + j0) = *reinterpret_cast<const uint4*>(h);
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (j0 + u < a.K) a.Vb[row * a.ldv + j0 + u] = __float2bfloat16_rn(v[u] - a.muR[j0 + u]);
        }
      } else if (row < a.n) {
        if (j0 + 7 < a.K) {
          float* dst = a.V + row * a.ldv + j0;
          const float4 m0 = __ldg(reinterpret_cast<const float4*>(a.muR + j0));
          const float4 m1 = __ldg(reinterpret_cast<const float4*>(a.muR + j0 + 4));
          reinterpret_cast<float4*>(dst)[0] = make_float4(v[0] - m0.x, v[1] - m0.y, v[2] - m0.z, v[3] - m0.w);
          reinterpret_cast<float4*>(dst)[1] = make_float4(v[4] - m1.x, v[5] - m1.y, v[6] - m1.z, v[7] - m1.w);
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (j0 + u < a.K) a.V[row * a.ldv + j0 + u] = v[u] - a.muR[j0 + u];
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // TMEM reads done before the next tile's MMAs overwrite it
  }
  if (!ok) {
    // let any MMA still in flight finish before releasing TMEM
    if (last_stage >= 0) {
      const uint32_t ul = last_stage ? uses1 : uses0;
      mbar_wait(&bars[last_stage], (ul - 1) & 1, kWaitIters);
    }
    if (tid == 0) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

int apply_tc_supported(int K) { return K >= 1 && K <= 511; }

size_t apply_tc_scratch_floats(int K) {
  const int Kq = (K + 15) & ~15, Kd = (K + 31) & ~31;
  return 2 * (size_t)Kq * Kd + Kq + 64;
}

hef_status apply_tc(void* V, bool bf16, long long ldv, long long n, int K, const float* Rinv, int Kp,
                    const float* mu, float* scratch, int* err, cudaStream_t st) {
  const int Kq = (K + 15) & ~15, Kd = (K + 31) & ~31;
  float* RtH = scratch;
  float* RtL = RtH + (size_t)Kq * Kd;
  float* muR = RtL + (size_t)Kq * Kd;
  HEF_LAUNCH("k_rinv_split", st, k_rinv_split<<<stride_grid((long long)Kq * Kd, 2), kThreads, 0, st>>>(
                                     Rinv, mu, K, Kp, Kq, Kd, RtH, RtL, muR));
  ApplyTcArgs a;
  a.V = bf16 ? nullptr : static_cast<float*>(V);
  a.Vb = bf16 ? static_cast<__nv_bfloat16*>(V) : nullptr;
  a.ldv = ldv;
  a.n = (int)n;
  a.K = K;
  a.Kq = Kq;
  a.Kd = Kd;
  a.RtH = RtH;
  a.RtL = RtL;
  a.muR = muR;
  a.err = err;
  const long long ntiles = (n + 127) / 128;
  const int ctas = (int)(ntiles < num_sms() ? ntiles : num_sms());
  const int nka = Kd / 32;
  const size_t bres = (size_t)(nka * Kq - 16 * nka * (nka - 1)) * 256;  // resident B, hi + lo
  const size_t smem_res = 1024 + bres + 2 * (2 * 128 * 128) + 64;
  const size_t stage = 2 * 128 * 128 + 2 * (size_t)Kq * 128;  // A and B of one K block
  const size_t smem2 = 1024 + 2 * stage + 64, smem1 = 1024 + stage + 64;
  auto launch = [&](auto kern, size_t smem) -> hef_status {
    HEF_ENSURE_SMEM(kern, (int)smem);
    HEF_LAUNCH("k_apply_tc", st, (kern<<<ctas, kApThreads, smem, st>>>(a)));
    return HEF_OK;
  };
  hef_status s;
  if (smem_res <= 220 * 1024)
    s = bf16 ? launch(k_apply_tc<true, 2, true>, smem_res) : launch(k_apply_tc<true, 2, false>, smem_res);
  else if (smem2 <= 220 * 1024)
    s = bf16 ? launch(k_apply_tc<false, 2, true>, smem2) : launch(k_apply_tc<false, 2, false>, smem2);
  else
    s = bf16 ? launch(k_apply_tc<false, 1, true>, smem1) : launch(k_apply_tc<false, 1, false>, smem1);
  if (s) return s;
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

int gram_tc_supported(int K) { return K >= 1 && K + 1 <= 512; }

int gram_tc_ctas(long long n) {
  long long want = (n + kSlab - 1) / kSlab;
  long long g = num_sms();
  return (int)(want < g ? (want > 0 ? want : 1) : g);
}

size_t gram_tc_part_doubles(long long n, int K) {
  const int Kq = (K + 1 + 15) & ~15;
  return (size_t)gram_tc_ctas(n) * Kq * Kq;
}

// Block rows of G_aug packed into CTA groups whose accumulators fit the 512
// TMEM columns (largest first, first fit).  Returns the number of groups.
static int gram_groups(int Kq, int nb, int (&gmask)[4]) {
  int load[4] = {0, 0, 0, 0};
  int ng = 0;
  for (int b = 0; b < nb; ++b) {
    const int N = Kq - 128 * b;
    int g = 0;
    while (g < ng && load[g] + N > 512) ++g;
    if (g == ng) gmask[ng++] = 0;
    gmask[g] |= 1 << b;
    load[g] += N;
  }
  return ng;
}

template <int NB, int STAGES>
static hef_status launch_gram_tc(const GramTcArgs& a, int ctas, int ng, cudaStream_t st) {
  const size_t smem = 1024 + 2 * (size_t)STAGES * NB * 128 * 128 + 64;
  if (a.Vb) {
    HEF_ENSURE_SMEM((k_gram_tc<NB, STAGES, true>), (int)smem);
    HEF_LAUNCH("k_gram_tc", st, (k_gram_tc<NB, STAGES, true><<<dim3(ctas, ng), kGrThreads, smem, st>>>(a)));
  } else {
    HEF_ENSURE_SMEM((k_gram_tc<NB, STAGES, false>), (int)smem);
    HEF_LAUNCH("k_gram_tc", st, (k_gram_tc<NB, STAGES, false><<<dim3(ctas, ng), kGrThreads, smem, st>>>(a)));
  }
  return HEF_OK;
}

hef_status gram_tc(const void* V, bool bf16, long long ldv, long long n, int K, double* part,
                   double* G, double* c, int* err, cudaStream_t st) {
  const int Kq = (K + 1 + 15) & ~15;
  const int nb = (Kq + 127) / 128;
  const int ctas = gram_tc_ctas(n);
  GramTcArgs a;
  a.V = bf16 ? nullptr : static_cast<const float*>(V);
  a.Vb = bf16 ? static_cast<const __nv_bfloat16*>(V) : nullptr;
  a.ldv = ldv;
  a.n = (int)n;
  a.K = K;
  a.Kq = Kq;
  a.nb = nb;
  a.rows_per_cta = (int)(((n + ctas - 1) / ctas + kSlab - 1) / kSlab * kSlab);
  a.part = reinterpret_cast<float*>(part);  // FP32 partials in the FP64-sized buffer
  a.err = err;
  for (int g = 0; g < 4; ++g) a.gmask[g] = 0;
  const int ng = gram_groups(Kq, nb, a.gmask);
  hef_status s;
  switch (nb) {
    case 1: s = launch_gram_tc<1, 2>(a, ctas, ng, st); break;
    case 2: s = launch_gram_tc<2, 2>(a, ctas, ng, st); break;
    case 3: s = launch_gram_tc<3, 2>(a, ctas, ng, st); break;
    default: s = launch_gram_tc<4, 1>(a, ctas, ng, st); break;
  }
  if (s) return s;
  HEF_LAUNCH("k_gram_tc_reduce", st,
             k_gram_tc_reduce<<<stride_grid(((long long)K * K + K) * 8, 8), kThreads, 0, st>>>(
                 reinterpret_cast<const float*>(part), K, Kq, ctas, G, c));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

}  // namespace hef
