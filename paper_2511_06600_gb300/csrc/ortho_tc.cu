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

#include <cstring>

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

// G (K x K, FP64) and c (K): fixed-order sums of the per-CTA FP32 partials of
// G_aug (column K holds the column sums), in double-float arithmetic (FP64
// operations are slow on this part; about 44 significant bits), rounded to
// FP64 at the end.  A block takes 32 consecutive entries (i, j), j in [i, K],
// of the row-major (K + 1)-wide upper part: warp w sums the partials w, w + 8,
// ... of its entries (each load a contiguous 128 bytes), then warp 0 adds the
// eight warp sums in warp order.
__global__ void __launch_bounds__(256) k_gram_tc_reduce(const float* __restrict__ part, int K, int Kq,
                                                        int nchunk, double* G, double* c) {
  __shared__ DFloat red[8][32];
  const int e = threadIdx.x & 31, sub = threadIdx.x >> 5;
  const long long total = (long long)K * (K + 1);
  const size_t stride = (size_t)Kq * Kq;
  for (long long base = (long long)blockIdx.x * 32; base < total; base += (long long)gridDim.x * 32) {
    const long long idx = base + e;
    const int i = (int)(idx / (K + 1)), j = (int)(idx % (K + 1));
    const bool act = idx < total && i <= j;
    DFloat s{0.f, 0.f};
    if (act) {
      const float* p = part + (size_t)i * Kq + j;
      int q = sub;
      for (; q + 56 < nchunk; q += 64) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (size_t)(q + 8 * u) * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) s = df_add(s, DFloat{v[u], 0.f});
      }
      for (; q < nchunk; q += 8) s = df_add(s, DFloat{__ldcg(p + (size_t)q * stride), 0.f});
    }
    red[sub][e] = s;
    __syncthreads();
    if (sub == 0 && act) {
      DFloat t = red[0][e];
#pragma unroll
      for (int u = 1; u < 8; ++u) t = df_add(t, red[u][e]);
      const double sd = (double)t.hi + (double)t.lo;
      if (j < K) {
        G[(size_t)i * K + j] = sd;
        G[(size_t)j * K + i] = sd;
      } else {
        c[i] = sd;
      }
    }
    __syncthreads();
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
  // muR[j] by a warp per column: lanes stride over i <= j, then a shuffle tree
  const int lane = threadIdx.x & 31;
  for (long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < Kq;
       j += ((long long)gridDim.x * blockDim.x) >> 5) {
    float s = 0.f;
    if (j < K)
      for (int i = lane; i <= (int)j; i += 32) s += mu[i] * Rinv[(size_t)i * Kp + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) muR[j] = s;
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

// ---------------------------------------------------------------- TMA pipelines
//
// The FP32 basis with a 16-byte aligned row pitch: tensor-map loads feed a
// warp-specialised pipeline, so that no warp waits for its own global loads.
//   warp 0            one thread issues the TMA loads into a ring of stages
//   warp 1            one thread issues the MMAs (tcgen05) and commits
//   converter warps   hi/lo TF32 split of each landed stage
//   epilogue warps    TMEM -> registers -> global memory (apply)
// Hand-offs are mbarriers; every wait is bounded (a timeout sets *err, and
// each role still waits for the copies and MMAs it issued before the CTA
// leaves).

constexpr int kTmThreads = 512;
constexpr int kTmConvFirst = 2;  // apply: warps 2..7 split, warps 8..15 drain
constexpr int kTmConvWarps = 6;
constexpr int kTmEpiFirst = 8;
constexpr int kTmEpiWarps = 8;
constexpr uint32_t kATile = 128u * 128u;  // one apply A tile: 128 rows x 32 values

struct ApplyTmaArgs {
  float* V;
  long long ldv;
  int n, K, Kq, Kd;
  const float* RtH;
  const float* RtL;
  const float* muR;
  int* err;
};

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, kWaitIters));
}

// Q = (V - 1 mu^T) Rinv in place, 128-row tiles (as k_apply_tc, RESB): the
// A tile of K block ka is the box (32 values from 32 ka) x (128 rows) of V,
// loaded K-major with the 128-byte swizzle, i.e. already in the MMA's
// layout; the converters round it to its hi part in place and write the lo
// part into one of two lo buffers (so that a stage holds 16 KB).  Two TMEM
// accumulators: tile t drains while tile t + 1 accumulates.  NS stages of A.
template <int NS>
__global__ void __launch_bounds__(kTmThreads, 1)
    k_apply_tma(ApplyTmaArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nka = a.Kd / 32;
  auto brows = [&](int ka) { return a.Kq - 32 * ka; };
  auto boff = [&](int ka) { return (uint32_t)(ka * a.Kq - 16 * ka * (ka - 1)) * 256u; };
  unsigned char* abase = base + boff(nka);          // stage s at s kATile
  unsigned char* lbase = abase + (uint32_t)NS * kATile;  // lo buffer b at b kATile
  uint64_t* full = reinterpret_cast<uint64_t*>(lbase + 2u * kATile);  // NS: landed
  uint64_t* conv = full + NS;     // NS: split
  uint64_t* empty = conv + NS;    // NS: MMAs done with the stage
  uint64_t* tfull = empty + NS;   // 2: accumulator complete
  uint64_t* tempty = tfull + 2;   // 2: accumulator drained
  uint64_t* lfree = tempty + 2;   // 2: MMAs done with the lo buffer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(lfree + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t ncols = 32;
  while (ncols < 2u * (uint32_t)a.Kq) ncols <<= 1;
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&conv[q], kTmConvWarps);
      mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kTmEpiWarps);
      mbar_init(&lfree[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // resident B tiles: tile ka holds rows 32 ka .. Kq - 1 of Rinv^T, basis
  // values [32 ka, 32 ka + 32)
  for (int ka = 0; ka < nka; ++ka) {
    unsigned char* bhi = base + boff(ka);
    unsigned char* blo = bhi + (uint32_t)brows(ka) * 128u;
    const int c0 = ka * 32;
    for (int f = tid; f < brows(ka) * 8; f += kTmThreads) {
      const int jr = f >> 3, q = f & 7;
      const size_t src = (size_t)(c0 + jr) * a.Kd + c0 + 4 * q;
      const uint32_t off = sw128_offset(jr, 4 * q);
      *reinterpret_cast<float4*>(bhi + off) = __ldg(reinterpret_cast<const float4*>(a.RtH + src));
      *reinterpret_cast<float4*>(blo + off) = __ldg(reinterpret_cast<const float4*>(a.RtL + src));
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = (a.n + 127) / 128;
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
        for (int ka = 0; ka < nka; ++ka) {
          const int s = g % NS;
          if (g >= NS && !(ok = mbar_wait(&empty[s], (uint32_t)((g / NS) - 1) & 1u, kWaitIters))) break;
          mbar_arrive_expect_tx(&full[s], kATile);
          tma_load_2d(abase + (uint32_t)s * kATile, &tmap, 32 * ka, tile * 128, &full[s]);
          ++g;
        }
      // copies still landing finish before the CTA may leave
      for (int q = g - NS > 0 ? g - NS : 0; q < g; ++q)
        mbar_wait(&full[q % NS], (uint32_t)(q / NS) & 1u, kWaitIters);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0, lt = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        const int b = lt & 1;
        if (lt >= 2 && !(ok = mbar_wait(&tempty[b], (uint32_t)((lt >> 1) - 1) & 1u, kWaitIters))) break;
        tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)(b * a.Kq);
        for (int ka = 0; ka < nka; ++ka, ++g) {
          const int s = g % NS;
          if (!(ok = mbar_wait(&conv[s], (uint32_t)(g / NS) & 1u, kWaitIters))) break;
          tc_fence_after();
          const int c0 = ka * 32, nr = brows(ka);
          const uint32_t sah = smem_u32(abase + (uint32_t)s * kATile);
          const uint32_t sal = smem_u32(lbase + (uint32_t)(g & 1) * kATile);
          const uint32_t sbh = smem_u32(base + boff(ka)), sbl = sbh + (uint32_t)nr * 128u;
          const uint32_t id = idesc_tf32(128, nr);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t ko = (uint32_t)ks * 32u;
            const uint32_t d = dbase + (uint32_t)c0;
            const uint32_t acc = (ka > 0 || ks > 0) ? 1u : 0u;  // block 0 starts every column
            mma_tf32(d, desc_k_sw128(sah + ko), desc_k_sw128(sbh + ko), id, acc);
            mma_tf32(d, desc_k_sw128(sah + ko), desc_k_sw128(sbl + ko), id, 1u);
            mma_tf32(d, desc_k_sw128(sal + ko), desc_k_sw128(sbh + ko), id, 1u);
          }
          mma_commit(&empty[s]);
          mma_commit(&lfree[g & 1]);
        }
        if (!ok) break;
        mma_commit(&tfull[b]);
      }
      // MMAs in flight finish before TMEM may be released
      if (g > 0) mbar_wait(&empty[(g - 1) % NS], (uint32_t)((g - 1) / NS) & 1u, kWaitIters);
    }
  } else if (warp < kTmEpiFirst) {
    const int ctid = tid - kTmConvFirst * 32;
    int g = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
      for (int ka = 0; ka < nka; ++ka, ++g) {
        const int s = g % NS;
        if (!(ok = warp_wait(&full[s], (uint32_t)(g / NS) & 1u))) break;
        if (g >= 2 && !(ok = warp_wait(&lfree[g & 1], (uint32_t)((g >> 1) - 1) & 1u))) break;
        float4* hi = reinterpret_cast<float4*>(abase + (uint32_t)s * kATile);
        float4* lo = reinterpret_cast<float4*>(lbase + (uint32_t)(g & 1) * kATile);
        for (int f = ctid; f < (int)(kATile / 16); f += kTmConvWarps * 32) {
          const float4 x = hi[f];
          const float4 h = make_float4(tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w));
          hi[f] = h;
          lo[f] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
      }
  } else {
    // warp w drains TMEM lanes 32 (w mod 4) ..; the two warps of a lane
    // quarter take alternate groups of 8 columns
    const int q4 = warp & 3, half = (warp - kTmEpiFirst) >> 2;
    int lt = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
      const int b = lt & 1;
      if (!(ok = warp_wait(&tfull[b], (uint32_t)(lt >> 1) & 1u))) break;
      tc_fence_after();
      const long long row = (long long)tile * 128 + q4 * 32 + lane;
      for (int c8 = half; c8 < a.Kq / 8; c8 += 2) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * a.Kq + c8 * 8), v);
        tmem_wait_ld();
        const int j0 = c8 * 8;
        if (row < a.n) {
          float* dst = a.V + row * a.ldv + j0;
          if (j0 + 7 < a.K) {
            const float4 m0 = __ldg(reinterpret_cast<const float4*>(a.muR + j0));
            const float4 m1 = __ldg(reinterpret_cast<const float4*>(a.muR + j0 + 4));
            reinterpret_cast<float4*>(dst)[0] = make_float4(v[0] - m0.x, v[1] - m0.y, v[2] - m0.z, v[3] - m0.w);
            reinterpret_cast<float4*>(dst)[1] = make_float4(v[4] - m1.x, v[5] - m1.y, v[6] - m1.z, v[7] - m1.w);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (j0 + u < a.K) dst[u] = v[u] - a.muR[j0 + u];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  if (!ok) atomicExch(a.err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

struct GramTmaArgs {
  int n, K, Kq, ncb;
  int rows_per_cta;
  int gmask[4];
  float* part;
  int* err;
};

// G_aug = [V 1]^T [V 1] (as k_gram_tc, NB <= 2 blocks of 128 basis rows).  A
// 32-row slab of V lands as ncb unswizzled boxes of 32 values x 32 rows in a
// ring of NR raw stages (only the converters read them); the converter warps
// (2..15) transpose it into the hi/lo K-major tiles of one of two tile
// stages, adding the ones column.
template <int NB, int NR>
__global__ void __launch_bounds__(kTmThreads, 1)
    k_gram_tma(GramTmaArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int Mpad = NB * 128;
  constexpr uint32_t tile_bytes = (uint32_t)Mpad * 128u;
  constexpr int kConv = kTmThreads / 32 - kTmConvFirst;  // converter warps
  const uint32_t raw_bytes = (uint32_t)a.ncb * 4096u;
  unsigned char* tiles = base;                            // stage u: hi, lo
  unsigned char* raw = base + 4u * tile_bytes;            // NR stages
  uint64_t* rfull = reinterpret_cast<uint64_t*>(raw + (size_t)NR * raw_bytes);
  uint64_t* rempty = rfull + NR;   // NR: converted out of
  uint64_t* tfull = rempty + NR;   // 2: tile stage written
  uint64_t* tempty = tfull + 2;    // 2: MMAs done with the tile stage
  uint64_t* done = tempty + 2;     // 1: every MMA complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gmask = a.gmask[blockIdx.y];
  int toff[NB];
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
    for (int q = 0; q < NR; ++q) {
      mbar_init(&rfull[q], 1);
      mbar_init(&rempty[q], kConv);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(&tfull[u], kConv);
      mbar_init(&tempty[u], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // basis rows [Kq, Mpad) of the tiles stay zero
  for (int q = 0; q < 4; ++q) {
    unsigned char* tile = tiles + (size_t)q * tile_bytes;
    for (int e = tid; e < (Mpad - a.Kq) * 32; e += kTmThreads)
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
  if (warp == 0) {
    if (lane == 0) {
      int t = 0;
      for (; t < nslab; ++t) {
        const int s = t % NR;
        if (t >= NR && !(ok = mbar_wait(&rempty[s], (uint32_t)((t / NR) - 1) & 1u, kWaitIters))) break;
        mbar_arrive_expect_tx(&rfull[s], raw_bytes);
        for (int cb = 0; cb < a.ncb; ++cb)
          tma_load_2d(raw + (size_t)s * raw_bytes + cb * 4096u, &tmap, 32 * cb, (int)(r0 + (long long)t * kSlab),
                      &rfull[s]);
      }
      for (int q = t - NR > 0 ? t - NR : 0; q < t; ++q)
        mbar_wait(&rfull[q % NR], (uint32_t)(q / NR) & 1u, kWaitIters);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int t = 0; t < nslab; ++t) {
        const int u = t & 1;
        if (!(ok = mbar_wait(&tfull[u], (uint32_t)(t >> 1) & 1u, kWaitIters))) break;
        tc_fence_after();
        const uint32_t shi = smem_u32(tiles + 2u * u * tile_bytes), slo = shi + tile_bytes;
#pragma unroll
        for (int ks = 0; ks < kSlab / 8; ++ks) {
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            if (!((gmask >> b) & 1)) continue;
            const int Nb = a.Kq - 128 * b;  // <= 256
            // block b: basis rows [128 b, 128 b + 128) against columns [128 b, Kq)
            const uint32_t aoff = (uint32_t)b * 128u * 128u + (uint32_t)ks * 32u;
            const uint32_t acc = (t > 0 || ks > 0) ? 1u : 0u;
            const uint32_t d = tmem + (uint32_t)toff[b];
            const uint32_t id = idesc_tf32(128, Nb);
            mma_tf32(d, desc_k_sw128(shi + aoff), desc_k_sw128(shi + aoff), id, acc);
            mma_tf32(d, desc_k_sw128(shi + aoff), desc_k_sw128(slo + aoff), id, 1u);
            mma_tf32(d, desc_k_sw128(slo + aoff), desc_k_sw128(shi + aoff), id, 1u);
          }
        }
        mma_commit(&tempty[u]);
      }
      mma_commit(done);
      if (!mbar_wait(done, 0u, kWaitIters)) ok = false;
    }
  } else {
    // warp item (column block cbw of 32 basis values, row half h): lane
    // (q = lane / 8, l = lane % 8) transposes the 4 x 4 block of slab rows
    // 4 rho .. 4 rho + 3, rho = ((l / 2 + q) mod 4) + 4 h, and basis values
    // 4 cq .. 4 cq + 3, cq = 8 cbw + l: four 16-byte loads of the unswizzled
    // raw rows (a quarter warp reads eight distinct 16-byte bank groups) and
    // eight 16-byte stores into the swizzled tiles (group rho ^ (c mod 8),
    // again distinct over a quarter warp)
    const int cw = warp - kTmConvFirst;
    const int q = lane >> 3, l = lane & 7;
    const int nwi = 2 * ((a.Kq + 31) / 32);
    for (int t = 0; t < nslab; ++t) {
      const int s = t % NR, u = t & 1;
      if (!(ok = warp_wait(&rfull[s], (uint32_t)(t / NR) & 1u))) break;
      if (t >= 2 && !(ok = warp_wait(&tempty[u], (uint32_t)((t >> 1) - 1) & 1u))) break;
      const unsigned char* rs = raw + (size_t)s * raw_bytes;
      unsigned char* hi = tiles + 2u * u * tile_bytes;
      unsigned char* lo = hi + tile_bytes;
      const long long rowbase = r0 + (long long)t * kSlab;
      for (int wi = cw; wi < nwi; wi += kConv) {
        const int cbw = wi >> 1, h = wi & 1;
        const int cq = 8 * cbw + l;
        if (4 * cq >= a.Kq) continue;
        const int rb = 4 * ((((l >> 1) + q) & 3) + 4 * h);
        float4 x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          x[k] = cbw < a.ncb ? *reinterpret_cast<const float4*>(rs + cbw * 4096 + (rb + k) * 128 + l * 16)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        float one[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) one[k] = rowbase + rb + k < a.n ? 1.f : 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int c = 4 * cq + w;
          float v[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float xv = w == 0 ? x[k].x : w == 1 ? x[k].y : w == 2 ? x[k].z : x[k].w;
            v[k] = c < a.K ? xv : (c == a.K ? one[k] : 0.f);
          }
          float hv[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) hv[k] = tf32_round(v[k]);
          const uint32_t off = sw128_offset(c, rb);
          *reinterpret_cast<float4*>(hi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<float4*>(lo + off) =
              make_float4(v[0] - hv[0], v[1] - hv[1], v[2] - hv[2], v[3] - hv[3]);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&rempty[s]);
        mbar_arrive(&tfull[u]);
      }
    }
  }
  // every MMA complete (the MMA thread's final commit) before TMEM is read
  if (warp != 1) ok = warp_wait(done, 0u) && ok;
  ok = __syncthreads_and(ok);
  tc_fence_after();
  float* P = a.part + (size_t)blockIdx.x * a.Kq * a.Kq;
  if (ok && nslab > 0) {
    const int q = warp & 3, part = warp >> 2;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!((gmask >> b) & 1)) continue;
      const int ncol = a.Kq - 128 * b;
      const int i = b * 128 + q * 32 + lane;
      for (int c8 = part; c8 < ncol / 8; c8 += kTmThreads / 128) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)toff[b] + (uint32_t)c8 * 8u, v);
        tmem_wait_ld();
        const int j0 = b * 128 + c8 * 8;
        if (i < a.Kq && j0 + 7 >= i) {
#pragma unroll
          for (int w = 0; w < 8; ++w) P[(size_t)i * a.Kq + j0 + w] = v[w];
        }
      }
    }
  } else {
    for (int e = tid; e < a.Kq * a.Kq; e += kTmThreads)
      if ((gmask >> ((e / a.Kq) / 128)) & 1) P[e] = 0.f;
    if (!ok && tid == 0) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

// Rows of a 4-byte basis that a tensor map can address: 16-byte aligned base
// and row pitch.
static bool tma_rows_ok(const void* V, long long ldv) {
  return (reinterpret_cast<uintptr_t>(V) & 15) == 0 && ((size_t)ldv * 4) % 16 == 0 && ldv <= (1ll << 36);
}

// Tensor map of the FP32 matrix V (n rows of K values, pitch ldv) with a box
// of bw values x bh rows (bw * 4 = 128 bytes), in the 128-byte swizzle or
// unswizzled; values past K and rows past n read as zero.
static bool encode_box_map(CUtensorMap* tm, const float* V, long long ldv, int K, long long n, int bw,
                           int bh, bool swizzle) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn || n < 1 || n > 0x7fffffffll || K < 1) return false;
  memset(tm, 0, sizeof(*tm));
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ldv * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(V), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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
  {
    // TMA pipeline: FP32 basis, 16-byte aligned rows, two accumulators of
    // Kq columns in TMEM, resident B and at least two A stages in shared memory
    const size_t bres_t = (size_t)(nka * Kq - 16 * nka * (nka - 1)) * 256;
    auto smem_tma = [&](int ns) { return 1024 + bres_t + (size_t)(ns + 2) * 128 * 128 + (3 * ns + 6) * 8 + 16; };
    CUtensorMap tm;
    if (!bf16 && Kq <= 256 && smem_tma(2) <= 227 * 1024 && tma_rows_ok(V, ldv) &&
        encode_box_map(&tm, static_cast<const float*>(V), ldv, K, n, 32, 128, true)) {
      ApplyTmaArgs t;
      t.V = static_cast<float*>(V);
      t.ldv = ldv;
      t.n = (int)n;
      t.K = K;
      t.Kq = Kq;
      t.Kd = Kd;
      t.RtH = RtH;
      t.RtL = RtL;
      t.muR = muR;
      t.err = err;
      if (smem_tma(4) <= 227 * 1024) {
        HEF_ENSURE_SMEM(k_apply_tma<4>, (int)smem_tma(4));
        HEF_LAUNCH("k_apply_tc", st, (k_apply_tma<4><<<ctas, kTmThreads, smem_tma(4), st>>>(t, tm)));
      } else if (smem_tma(3) <= 227 * 1024) {
        HEF_ENSURE_SMEM(k_apply_tma<3>, (int)smem_tma(3));
        HEF_LAUNCH("k_apply_tc", st, (k_apply_tma<3><<<ctas, kTmThreads, smem_tma(3), st>>>(t, tm)));
      } else {
        HEF_ENSURE_SMEM(k_apply_tma<2>, (int)smem_tma(2));
        HEF_LAUNCH("k_apply_tc", st, (k_apply_tma<2><<<ctas, kTmThreads, smem_tma(2), st>>>(t, tm)));
      }
      HEF_CHECK_LAUNCH();
      return HEF_OK;
    }
  }
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
  CUtensorMap tm;
  const int ncb = (K + 31) / 32;
  // TMA pipeline: FP32 basis, 16-byte aligned rows, at most two blocks of
  // 128 basis rows, two tile stages and at least two raw stages in shared memory
  auto smem_tma = [&](int nr) {
    return 1024 + 4 * (size_t)nb * 128 * 128 + (size_t)nr * ncb * 4096 + (2 * nr + 5) * 8 + 16;
  };
  if (!bf16 && nb <= 2 && smem_tma(2) <= 227 * 1024 && tma_rows_ok(V, ldv) &&
      encode_box_map(&tm, static_cast<const float*>(V), ldv, K, n, 32, kSlab, false)) {
    GramTmaArgs t;
    t.n = (int)n;
    t.K = K;
    t.Kq = Kq;
    t.ncb = ncb;
    t.rows_per_cta = a.rows_per_cta;
    for (int g = 0; g < 4; ++g) t.gmask[g] = a.gmask[g];
    t.part = a.part;
    t.err = err;
    int nr = 4;
    while (nr > 2 && smem_tma(nr) > 227 * 1024) --nr;
    const dim3 grid(ctas, ng);
#define HEF_GRAM_TMA(NBv, NRv)                                                                  \
  do {                                                                                          \
    HEF_ENSURE_SMEM((k_gram_tma<NBv, NRv>), (int)smem_tma(NRv));                                \
    HEF_LAUNCH("k_gram_tc", st,                                                                 \
               (k_gram_tma<NBv, NRv><<<grid, kTmThreads, smem_tma(NRv), st>>>(t, tm)));         \
  } while (0)
    if (nb == 1) {
      if (nr == 4) HEF_GRAM_TMA(1, 4);
      else if (nr == 3) HEF_GRAM_TMA(1, 3);
      else HEF_GRAM_TMA(1, 2);
    } else {
      if (nr == 4) HEF_GRAM_TMA(2, 4);
      else if (nr == 3) HEF_GRAM_TMA(2, 3);
      else HEF_GRAM_TMA(2, 2);
    }
#undef HEF_GRAM_TMA
    s = HEF_OK;
  } else {
    switch (nb) {
    case 1: s = launch_gram_tc<1, 2>(a, ctas, ng, st); break;
    case 2: s = launch_gram_tc<2, 2>(a, ctas, ng, st); break;
    case 3: s = launch_gram_tc<3, 2>(a, ctas, ng, st); break;
    default: s = launch_gram_tc<4, 1>(a, ctas, ng, st); break;
    }
  }
  if (s) return s;
  HEF_LAUNCH("k_gram_tc_reduce", st,
             k_gram_tc_reduce<<<(int)std::min<long long>(((long long)K * (K + 1) + 31) / 32, 8ll * num_sms()), 256, 0, st>>>(
                 reinterpret_cast<const float*>(part), K, Kq, ctas, G, c));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

}  // namespace hef
