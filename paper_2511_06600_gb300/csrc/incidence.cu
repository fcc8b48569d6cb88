// Incidence build: Algorithm 1 steps 1-2 (star and clique expansions of
// Section III-A.3, kept implicit).  Validates H on the device, orders the
// hyperedges for locality (ascending smallest pin, stable), builds the
// vertex-major transpose with a stable counting sort (so every later sum runs
// in a fixed order) and the per-edge / per-vertex scalars of both expansions.
// The device-wide scan and the LSD radix sort here serve the downstream
// level (sort of R).
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace hef {

namespace {

constexpr int kItems = 8;                      // items per thread (scan/sort)
constexpr int kTile = kThreads * kItems;        // 2048 items per tile

// ----------------------------------------------------------------- scan

// Single-pass scan (decoupled look-back): tiles of kScanTile items, each CTA
// takes the next tile id from an atomic counter (so a tile waits only on
// tiles that running CTAs have claimed), publishes its aggregate, then warp 0
// looks back over up to 32 predecessors at a time (aggregates summed until
// the nearest published prefix) and publishes its inclusive prefix.  Status
// word of tile t: high half 0 empty, 1 aggregate, 2 prefix; low half the
// value.  Bounded waits set HEF_WAIT_TIMEOUT in *err (when given).
constexpr int kScanThreads = 1024;
constexpr int kScanTile = kScanThreads * kItems;  // 8192
constexpr unsigned int kScanWaitIters = 1u << 22;

__device__ __forceinline__ int block_exclusive_scan_1024(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int q = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, q, o);
      if (lane >= o) q += y;
    }
    wsum[lane] = q;
  }
  __syncthreads();
  const int incl = x + (wid ? wsum[wid - 1] : 0);
  *total = wsum[31];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan1(const int* in, int* out, int N, int ntiles,
                                                        unsigned int* tctr,
                                                        unsigned long long* stat,
                                                        unsigned int* err) {
  __shared__ int s_tile, s_excl;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(tctr, 1u);
  __syncthreads();
  const int t = s_tile;
  const long long base = (long long)t * kScanTile + (long long)threadIdx.x * kItems;
  int v[kItems];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    v[j] = base + j < N ? in[base + j] : 0;
    sum += v[j];
  }
  int total;
  const int local = block_exclusive_scan_1024(sum, &total);
  if (ntiles > 1 && threadIdx.x < 32) {  // one tile: nothing to publish or look back on
    const int lane = threadIdx.x;
    if (lane == 0) {
      const unsigned long long w = ((t == 0 ? 2ull : 1ull) << 32) | (unsigned int)total;
      asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(stat + t), "l"(w) : "memory");
    }
    int excl = 0;
    for (int p = t - 1; p >= 0;) {
      const int q = p - lane;
      unsigned long long w = 2ull << 32;  // before tile 0: a zero prefix
      if (q >= 0) {
        unsigned int it = 0;
        do {
          asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(stat + q) : "memory");
        } while ((w >> 32) == 0ull && ++it < kScanWaitIters);
        if ((w >> 32) == 0ull && err) atomicOr(err, HEF_WAIT_TIMEOUT);
      }
      const unsigned pm = __ballot_sync(0xffffffffu, (w >> 32) == 2ull);
      const int lp = pm ? __ffs(pm) - 1 : 32;  // nearest published prefix
      int val = (lane <= lp && q >= 0) ? (int)(unsigned int)(w & 0xffffffffull) : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
      excl += val;
      if (lp < 32) break;
      p -= 32;
    }
    if (lane == 0) {
      if (t > 0) {
        const unsigned long long w = (2ull << 32) | (unsigned int)(excl + total);
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(stat + t), "l"(w) : "memory");
      }
      s_excl = excl;
    }
  } else if (threadIdx.x == 0) {
    s_excl = 0;
  }
  __syncthreads();
  int run = s_excl + local;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    if (base + j < N) out[base + j] = run;
    run += v[j];
  }
  if (t == ntiles - 1 && threadIdx.x == 0) out[N] = s_excl + total;
}

}  // namespace

int scan_tiles(long long N) { return (int)((N + kTile - 1) / kTile); }

// out[0..N] = exclusive scan of in[0..N); out[N] = total (k_scan1).  bsum
// needs scan_tiles(N) + 1 ints; counter is zero on entry (and on exit).  `in`
// and `out` may alias.
hef_status exclusive_scan(const int* in, int* out, long long N, int* bsum, unsigned int* counter,
                          cudaStream_t st, unsigned int* err) {
  (void)counter;  // the single-pass scan keeps its tile counter in bsum
  if (N == 0) {
    HEF_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(int), st));
    return HEF_OK;
  }
  // bsum (scan_tiles(N) + 1 ints, 8-byte aligned) holds the tile counter and,
  // for more than one tile, a 64-bit status word per kScanTile tile:
  // 2 + 2 ceil(N / 8192) ints, which then never exceeds it
  const int nt = (int)((N + kScanTile - 1) / kScanTile);
  HEF_CHECK_CUDA(cudaMemsetAsync(bsum, 0, (size_t)(nt == 1 ? 1 : 2 + 2 * nt) * sizeof(int), st));
  HEF_LAUNCH("k_scan1", st, k_scan1<<<nt, kScanThreads, 0, st>>>(
                                in, out, (int)N, nt, reinterpret_cast<unsigned int*>(bsum),
                                reinterpret_cast<unsigned long long*>(bsum + 2), err));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

namespace {

// ----------------------------------------------------------------- stable LSD radix sort (downstream sort of R)

// Digits of up to kMaxDigitBits bits: keys of b bits take ceil(b / 10)
// passes of equal width (an 18-bit vertex id: two passes of 9 bits).
constexpr int kMaxDigitBits = 10;
constexpr int kMaxBuckets = 1 << kMaxDigitBits;

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int N, int shift, int nb,
                             int* __restrict__ counts, int ntiles) {
  __shared__ int hist[kMaxBuckets];
  for (int d = threadIdx.x; d < nb; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  const uint32_t mask = (uint32_t)nb - 1u;
  const long long base = (long long)blockIdx.x * kTile;
  for (int j = 0; j < kItems; ++j) {
    long long i = base + (long long)j * kThreads + threadIdx.x;
    if (i < N) atomicAdd(&hist[(keys[i] >> shift) & mask], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nb; d += blockDim.x) counts[d * ntiles + blockIdx.x] = hist[d];
}

// Stable scatter: items are visited in index order (striped over threads),
// and each item's rank counts the earlier items of its tile with the same
// digit (warp match + per-warp digit counts).
__global__ void k_radix_scatter(const uint32_t* __restrict__ keys, const int32_t* __restrict__ vals,
                                int N, int shift, int nb, const int* __restrict__ offs, int ntiles,
                                uint32_t* __restrict__ okeys, int32_t* __restrict__ ovals) {
  __shared__ int base[kMaxBuckets];
  __shared__ int wcnt[kThreads / 32][kMaxBuckets];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t mask = (uint32_t)nb - 1u;
  for (int d = threadIdx.x; d < nb; d += blockDim.x) base[d] = offs[d * ntiles + blockIdx.x];
  const long long tile0 = (long long)blockIdx.x * kTile;
  for (int j = 0; j < kItems; ++j) {
    for (int d = threadIdx.x; d < nb; d += blockDim.x)
      for (int w = 0; w < kThreads / 32; ++w) wcnt[w][d] = 0;
    __syncthreads();
    long long i = tile0 + (long long)j * kThreads + threadIdx.x;
    bool valid = i < N;
    uint32_t key = valid ? keys[i] : 0u;
    int digit = valid ? (int)((key >> shift) & mask) : nb;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[wid][digit] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over warps, then advance the running base
    for (int d = threadIdx.x; d < nb; d += blockDim.x) {
      int run = base[d];
      for (int w = 0; w < kThreads / 32; ++w) {
        int c = wcnt[w][d];
        wcnt[w][d] = run;
        run += c;
      }
      base[d] = run;
    }
    __syncthreads();
    if (valid) {
      int pos = wcnt[wid][digit] + rank;
      okeys[pos] = key;
      ovals[pos] = vals[i];
    }
    __syncthreads();
  }
}

}  // namespace

void carve_sort_bufs(Carver& c, long long N, SortBufs* b) {
  const int ntiles = scan_tiles(N > 0 ? N : 1);
  b->k_alt = c.take<uint32_t>(N > 0 ? N : 1);
  b->v_alt = c.take<int32_t>(N > 0 ? N : 1);
  b->counts = c.take<int>((long long)kMaxBuckets * ntiles + 1);
  b->bsum = c.take<int>(scan_tiles((long long)kMaxBuckets * ntiles) + 1);
}

// Sorts (keys, vals) by key, stable; keys < 2^bits.  Result in keys/vals.
hef_status radix_sort(uint32_t* keys, int32_t* vals, long long N, int bits, SortBufs b,
                      cudaStream_t st) {
  if (N <= 1) return HEF_OK;
  const int ntiles = scan_tiles(N);
  const int npass = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
  const int dbits = (bits + npass - 1) / npass;
  const int nb = 1 << dbits;
  uint32_t* kin = keys;
  int32_t* vin = vals;
  uint32_t* kout = b.k_alt;
  int32_t* vout = b.v_alt;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += dbits, ++passes) {
    HEF_LAUNCH("k_radix_hist", st, k_radix_hist<<<ntiles, kThreads, 0, st>>>(kin, (int)N, shift, nb,
                                                                           b.counts, ntiles));
    HEF_CHECK_LAUNCH();
    hef_status s = exclusive_scan(b.counts, b.counts, (long long)nb * ntiles, b.bsum, b.counter, st);
    if (s) return s;
    HEF_LAUNCH("k_radix_scatter", st, k_radix_scatter<<<ntiles, kThreads, 0, st>>>(kin, vin, (int)N, shift, nb,
                                                                                 b.counts, ntiles, kout, vout));
    HEF_CHECK_LAUNCH();
    uint32_t* tk = kin; kin = kout; kout = tk;
    int32_t* tv = vin; vin = vout; vout = tv;
  }
  if (passes & 1) {
    HEF_CHECK_CUDA(cudaMemcpyAsync(keys, kin, N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    HEF_CHECK_CUDA(cudaMemcpyAsync(vals, vin, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  }
  return HEF_OK;
}

namespace {

// ----------------------------------------------------------------- build kernels

__device__ __forceinline__ void flag(unsigned int* status, unsigned bits, int e) {
  atomicOr(&status[0], bits);
  atomicMin(&status[1], (unsigned)e);
}

// Offsets, weight, pin range and duplicate pins of every hyperedge, and its
// locality key (smallest pin; 0 for an empty hyperedge) with val = caller id
// and the key's count in cnt:
// one thread per hyperedge, the pins of a hyperedge with at most kRegPins
// loaded at once into registers; its warp together for longer hyperedges,
// duplicates then found by a hash table in shared memory (quadratic scan
// beyond kHashSlots / 2 pins).
constexpr int kRegPins = 8;
constexpr int kHashSlots = 1024;  // per warp: duplicate checks of up to 512 pins in O(k)

__global__ void k_validate(int n, int m, long long P, const int64_t* __restrict__ eptr,
                           const int32_t* __restrict__ pins, const double* __restrict__ w,
                           unsigned int* status, uint32_t* keys, int32_t* vals, int* cnt) {
  __shared__ int htab[kThreads / 32][kHashSlots];
  const int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (eptr[0] != 0 || eptr[m] != P) flag(status, HEF_BAD_EPTR, 0);
  }
  for (long long base = (long long)blockIdx.x * blockDim.x; base < m;
       base += (long long)gridDim.x * blockDim.x) {
    const long long e = base + threadIdx.x;
    long long a = 0, b = 0;
    bool big = false;
    int mn = 0x7fffffff;
    if (e < m) {
      a = eptr[e], b = eptr[e + 1];
      if (a < 0 || b < a || b > P) {
        flag(status, HEF_BAD_EPTR, (int)e);
        a = b = 0;
      }
      const double we = w[e];
      if (!(we > 0.0 && we <= 1.7976931348623157e308)) flag(status, HEF_BAD_WEIGHT, (int)e);
      const int k = (int)(b - a);
      bool bad_pin = false, dup = false;
      if (k > kRegPins) {
        big = true;
      } else if (k > 0) {
        int q[kRegPins];
#pragma unroll
        for (int i = 0; i < kRegPins; ++i) q[i] = pins[a + min(i, k - 1)];
#pragma unroll
        for (int i = 0; i < kRegPins; ++i) {
          if (i < k) {
            bad_pin |= q[i] < 0 || q[i] >= n;
            mn = min(mn, q[i]);
#pragma unroll
            for (int j = i + 1; j < kRegPins; ++j) dup |= j < k && q[j] == q[i];
          }
        }
      }
      if (bad_pin) flag(status, HEF_BAD_PIN, (int)e);
      if (dup) flag(status, HEF_DUP_PIN, (int)e);
    }
    unsigned mask = __ballot_sync(0xffffffffu, big);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const long long ba = __shfl_sync(0xffffffffu, a, src), bb = __shfl_sync(0xffffffffu, b, src);
      const int k = (int)(bb - ba);
      bool bad_pin = false, dup = false;
      int wmn = 0x7fffffff;
      if (k <= kHashSlots / 2) {
        // duplicates by insertion into an open-addressing table of at least
        // 2k slots in shared memory (linear probing, multiplicative hash)
        int bits = 1;
        while ((1 << bits) < 2 * k) ++bits;
        const unsigned hmask = (1u << bits) - 1u;
        int* tab = htab[threadIdx.x >> 5];
        for (int i = lane; i <= (int)hmask; i += 32) tab[i] = -1;
        __syncwarp();
        for (int i = lane; i < k; i += 32) {
          const int p = pins[ba + i];
          wmn = min(wmn, p);
          if (p < 0 || p >= n) {
            bad_pin = true;
            continue;
          }
          unsigned h = ((unsigned)p * 2654435761u) >> (32 - bits);
          while (true) {
            const int old = atomicCAS(&tab[h], -1, p);
            if (old == -1) break;
            if (old == p) {
              dup = true;
              break;
            }
            h = (h + 1u) & hmask;
          }
        }
        __syncwarp();
      } else {
        for (int i = lane; i < k; i += 32) {
          const int p = pins[ba + i];
          if (p < 0 || p >= n) bad_pin = true;
          wmn = min(wmn, p);
          for (int j = i + 1; j < k; ++j)
            if (pins[ba + j] == p) dup = true;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wmn = min(wmn, __shfl_xor_sync(0xffffffffu, wmn, o));
      if (lane == src) mn = wmn;
      const long long ee = base + (threadIdx.x & ~31u) + src;
      if (__any_sync(0xffffffffu, bad_pin) && lane == 0) flag(status, HEF_BAD_PIN, (int)ee);
      if (__any_sync(0xffffffffu, dup) && lane == 0) flag(status, HEF_DUP_PIN, (int)ee);
    }
    if (e < m) {
      const uint32_t key = b > a ? (uint32_t)mn : 0u;
      keys[e] = key;
      vals[e] = (int32_t)e;
      if (key < (uint32_t)n) atomicAdd(&cnt[key], 1);  // bucket sizes of the locality sort
    }
  }
}

__global__ void k_edge_sizes(int m, const int64_t* __restrict__ eptr, const int32_t* __restrict__ sched,
                             const unsigned int* status, int* sizes) {
  if (status[0]) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    int e = sched[i];
    sizes[i] = (int)(eptr[e + 1] - eptr[e]);
  }
}

// Per internal hyperedge: pins in internal order, weights of both expansions,
// slot -> edge map, vertex incidence counts, and sum of w over |e| >= 2.
__global__ void k_edge_fill(int m, int clique_mode, const int64_t* __restrict__ eptr,
                            const int32_t* __restrict__ pins, const double* __restrict__ w,
                            const int32_t* __restrict__ sched, const int32_t* __restrict__ ceptr,
                            unsigned int* status, unsigned int* counter, int32_t* perm,
                            int32_t* cpins, int32_t* slot_edge, double* ew, double* ewh, double* ez,
                            float* f_ew, float* f_ewh, float* f_ez, double* ec, int* deg,
                            double* part, double* totals) {
  if (status[0]) return;
  double wsum = 0.0;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < m;
       base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    const bool valid = i < m;
    int e = 0, c0 = 0, k = 0;
    long long a = 0;
    if (valid) {
      e = sched[i];
      a = eptr[e];
      c0 = ceptr[i];
      k = ceptr[i + 1] - c0;
      perm[i] = e;
      if (k <= kRegPins) {  // pins loaded together, then stored
        int q[kRegPins];
#pragma unroll
        for (int t = 0; t < kRegPins; ++t) q[t] = t < k ? pins[a + t] : 0;
#pragma unroll
        for (int t = 0; t < kRegPins; ++t) {
          if (t < k) {
            cpins[c0 + t] = q[t];
            slot_edge[c0 + t] = (int32_t)i;
            atomicAdd(&deg[q[t]], 1);
          }
        }
      } else if (k <= 32) {
        for (int t = 0; t < k; ++t) {
          const int p = pins[a + t];
          cpins[c0 + t] = p;
          slot_edge[c0 + t] = (int32_t)i;
          atomicAdd(&deg[p], 1);
        }
      }
    }
    unsigned mask = __ballot_sync(0xffffffffu, valid && k > 32);
    while (mask) {  // long hyperedges: the warp copies their pins
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const long long sa = __shfl_sync(0xffffffffu, a, src);
      const int sc0 = __shfl_sync(0xffffffffu, c0, src), sk = __shfl_sync(0xffffffffu, k, src);
      for (int t = lane; t < sk; t += 32) {
        const int p = pins[sa + t];
        cpins[sc0 + t] = p;
        slot_edge[sc0 + t] = (int32_t)(base + (threadIdx.x & ~31u) + src);
        atomicAdd(&deg[p], 1);
      }
    }
    if (!valid) continue;
    const double we = w[e];
    double wa = 0.0, bh = 0.0, z = 0.0;
    if (k >= 2) {
      wa = we;
      bh = clique_mode == HEF_CLIQUE_PAPER ? we / (0.5 * (double)k * (double)(k - 1))
                                           : we / (double)(k - 1);
      z = we / (double)k;
      wsum += we;
    }
    ew[i] = wa, ewh[i] = bh, ez[i] = z;
    ec[i] = k >= 2 ? bh * (double)(k - 1) : 0.0;  // clique degree contribution, added per incidence
    f_ew[i] = (float)wa, f_ewh[i] = (float)bh, f_ez[i] = (float)z;
  }
  double v[1] = {wsum};
  block_partials<1>(v, part);
  if (last_block_done(counter)) {
    __shared__ double tot[1];
    reduce_slots(part, gridDim.x, 1, tot);
    if (threadIdx.x == 0) totals[2] = tot[0];
  }
}

// Window table: hyperedge e (thread, e in [0, m], ceptr[m] = P) is the first
// of the windows w with ceptr[e-1] < w kWinSlots <= ceptr[e]; the windows
// past ceptr[m] (only the last one when P is not a multiple) get m.
__global__ void k_windows(int m, long long P, const int32_t* __restrict__ ceptr,
                          const unsigned int* status, int32_t* win_edge) {
  if (status[0]) return;
  const long long nwin = num_windows(P);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e <= m;
       e += (long long)gridDim.x * blockDim.x) {
    const long long lo = e == 0 ? 0 : (long long)ceptr[e - 1] / kWinSlots + 1;
    const long long hi = e == m ? nwin : (long long)ceptr[e] / kWinSlots;
    for (long long w = lo; w <= hi && w <= nwin; ++w) win_edge[w] = (int32_t)e;
  }
}

// flags of hyperedges with more than kBigEdge pins (internal order)
__global__ void k_big_flags(int m, const int32_t* __restrict__ ceptr, const unsigned int* status,
                            int* flags) {
  if (status[0]) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x)
    flags[i] = (ceptr[i + 1] - ceptr[i]) > kBigEdge ? 1 : 0;
}

__global__ void k_big_scatter(int m, const int32_t* __restrict__ ceptr,
                              const int32_t* __restrict__ pos, const unsigned int* status,
                              int32_t* idx) {
  if (status[0]) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x)
    if ((ceptr[i + 1] - ceptr[i]) > kBigEdge) idx[pos[i]] = (int32_t)i;
}

// Stable counting sort of the indices i < N by keys[i] < nb (the locality
// schedule of hyperedges, the vertex-major transpose of the CSC slots): the
// bucket sizes come from atomics and an exclusive scan gives the offsets
// off[0..nb]; k_place drops each index into its bucket behind an atomic
// cursor (any order), and k_bucket_order sorts each bucket by index, which
// is the order a stable sort leaves: the result does not depend on
// scheduling.
__global__ void k_place(long long N, const int32_t* __restrict__ keys, const int32_t* __restrict__ off,
                        int* cur, const unsigned int* status, int32_t* placed) {
  if (status[0]) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = keys[i];
    placed[off[k] + atomicAdd(&cur[k], 1)] = (int32_t)i;
  }
}

constexpr int kSmallBucket = 8;  // buckets up to this size: one thread, a sorting network

// out[off[b] ..] = the indices of bucket b ascending (and out2[t] =
// map[out[t]] when map is given): one thread per bucket of at most
// kSmallBucket entries (an insertion network in registers), the bucket's warp
// for larger ones (each entry's rank is the count of smaller entries; the
// indices are distinct).
__global__ void k_bucket_order(long long nb, const int32_t* __restrict__ off,
                               const int32_t* __restrict__ placed, const int32_t* __restrict__ map,
                               const unsigned int* status, int32_t* out, int32_t* out2) {
  if (status[0]) return;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nb;
       base += (long long)gridDim.x * blockDim.x) {
    const long long b = base + threadIdx.x;
    int a0 = 0, d = 0;
    if (b < nb) a0 = off[b], d = off[b + 1] - a0;
    const bool big = d > kSmallBucket;
    if (d > 0 && !big) {
      int x[kSmallBucket];
#pragma unroll
      for (int q = 0; q < kSmallBucket; ++q) x[q] = q < d ? placed[a0 + q] : 0x7fffffff;
#pragma unroll
      for (int i = 1; i < kSmallBucket; ++i)
#pragma unroll
        for (int j = i; j > 0; --j) {
          const int lo = min(x[j - 1], x[j]), hi = max(x[j - 1], x[j]);
          x[j - 1] = lo, x[j] = hi;
        }
#pragma unroll
      for (int q = 0; q < kSmallBucket; ++q)
        if (q < d) {
          out[a0 + q] = x[q];
          if (map) out2[a0 + q] = map[x[q]];
        }
    }
    unsigned mask = __ballot_sync(0xffffffffu, big);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int s0 = __shfl_sync(0xffffffffu, a0, src), sd = __shfl_sync(0xffffffffu, d, src);
      for (int i = lane; i < sd; i += 32) {
        const int v = placed[s0 + i];
        int r = 0;
        for (int j = 0; j < sd; ++j) r += placed[s0 + j] < v ? 1 : 0;
        out[s0 + r] = v;
        if (map) out2[s0 + r] = map[v];
      }
    }
  }
}

// Vertex degrees of both expansions, in CSR (ascending hyperedge) order:
// d_c(v) = sum_e ewh_e (|e|-1), d_b(v) = sum_e w_e/|e|.
__global__ void k_node_scalars(int n, const int32_t* __restrict__ vptr, const int32_t* __restrict__ vedge,
                               const double* __restrict__ ec, const double* __restrict__ ewh,
                               const double* __restrict__ ez, unsigned int* status,
                               unsigned int* counter, double* dc, double* db, double* inv_dc,
                               double* inv_db, double* wsc, float* f_dc, float* f_db,
                               float* f_inv_dc, float* f_inv_db, float* f_wsc, double* part,
                               double* totals) {
  if (status[0]) return;
  double sc = 0.0, sb = 0.0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    double c = 0.0, b = 0.0, ws = 0.0;
    const int t0 = vptr[v], t1 = vptr[v + 1];
    // four incidences per round: their hyperedge ids, then their three
    // per-edge terms, each set of loads in flight together (sums in incidence
    // order; the clique term ewh_e (|e|-1) comes precomputed per hyperedge)
    for (int t = t0; t < t1; t += 4) {
      int e[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) e[u] = vedge[min(t + u, t1 - 1)];
      double wc[4], wh[4], wz[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        wc[u] = ec[e[u]];
        wh[u] = ewh[e[u]];
        wz[u] = ez[e[u]];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (t + u < t1) {
          c += wc[u];
          b += wz[u];
          ws += wh[u];
        }
      }
    }
    wsc[v] = ws;
    dc[v] = c;
    db[v] = b;
    inv_dc[v] = c > 0.0 ? 1.0 / c : 0.0;
    inv_db[v] = b > 0.0 ? 1.0 / b : 0.0;
    f_wsc[v] = (float)ws, f_dc[v] = (float)c, f_db[v] = (float)b;
    f_inv_dc[v] = (float)inv_dc[v], f_inv_db[v] = (float)inv_db[v];
    sc += c;
    sb += b;
  }
  double v2[2] = {sc, sb};
  block_partials<2>(v2, part);
  if (last_block_done(counter)) {
    __shared__ double tot[2];
    reduce_slots(part, gridDim.x, 2, tot);
    if (threadIdx.x < 2) totals[threadIdx.x] = tot[threadIdx.x];
  }
}

__global__ void k_export_vedge(long long P, const int32_t* __restrict__ vedge,
                               const int32_t* __restrict__ perm, int32_t* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = perm[vedge[i]];
}

// ----------------------------------------------------------------- workspace layout

struct IncLayout {
  hef_incidence h;
  uint32_t* keys;
  int32_t* vals;
  SortBufs sb;
  int* tmp;       // max(m, n) + 1 ints (sizes / degree counts, scanned in place)
  int* cur;       // max(m, n) + 1 ints: cursors of the counting sorts
  int32_t* place; // max(m, P): indices as placed in their buckets
  double* ec;     // m: ewh_e (|e| - 1), the clique-degree term of each hyperedge
  int* scan_bsum;
  double* part;
};

size_t carve_incidence(void* base, long long n, long long m, long long P, IncLayout* L) {
  Carver c(base);
  const long long NS = (m > P ? m : P);
  const long long NT = (m > n ? m : n) + 1;
  L->h.status = c.take<unsigned int>(64);
  L->h.counter = L->h.status + 32;
  L->sb.counter = L->h.status + 34;  // zeroed with the status word at the start of a build
  L->h.perm = c.take<int32_t>(m > 0 ? m : 1);
  L->h.ceptr = c.take<int32_t>(m + 1);
  L->h.cpins = c.take<int32_t>(P > 0 ? P : 1);
  L->h.slot_edge = c.take<int32_t>(P > 0 ? P : 1);
  L->h.big_idx = c.take<int32_t>(m > 0 ? m : 1);
  L->h.big_pos = c.take<int32_t>(m + 1);
  L->h.win_edge = c.take<int32_t>(num_windows(P) + 1);
  L->h.ew = c.take<double>(m > 0 ? m : 1);
  L->h.ewh = c.take<double>(m > 0 ? m : 1);
  L->h.ez = c.take<double>(m > 0 ? m : 1);
  L->h.vptr = c.take<int32_t>(n + 1);
  L->h.vedge = c.take<int32_t>(P > 0 ? P : 1);
  L->h.vslot = c.take<int32_t>(P > 0 ? P : 1);
  L->h.dc = c.take<double>(n > 0 ? n : 1);
  L->h.db = c.take<double>(n > 0 ? n : 1);
  L->h.inv_dc = c.take<double>(n > 0 ? n : 1);
  L->h.inv_db = c.take<double>(n > 0 ? n : 1);
  L->h.wsc = c.take<double>(n > 0 ? n : 1);
  L->h.f_ew = c.take<float>(m > 0 ? m : 1);
  L->h.f_ewh = c.take<float>(m > 0 ? m : 1);
  L->h.f_ez = c.take<float>(m > 0 ? m : 1);
  L->h.f_dc = c.take<float>(n > 0 ? n : 1);
  L->h.f_db = c.take<float>(n > 0 ? n : 1);
  L->h.f_inv_dc = c.take<float>(n > 0 ? n : 1);
  L->h.f_inv_db = c.take<float>(n > 0 ? n : 1);
  L->h.f_wsc = c.take<float>(n > 0 ? n : 1);
  L->h.totals = c.take<double>(8);
  L->keys = c.take<uint32_t>(NS > 0 ? NS : 1);
  L->vals = c.take<int32_t>(NS > 0 ? NS : 1);
  L->place = c.take<int32_t>(NS > 0 ? NS : 1);
  L->ec = c.take<double>(m > 0 ? m : 1);
  L->tmp = c.take<int>(NT);
  L->cur = c.take<int>(NT);
  L->scan_bsum = c.take<int>(scan_tiles(NT) + 1);
  L->part = c.take<double>(2ll * 8 * 1024);
  return c.bytes();
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" size_t hef_incidence_workspace_bytes(int64_t n, int64_t m, int64_t P) {
  if (n < 0 || m < 0 || P < 0) return 0;
  IncLayout L;
  return carve_incidence(nullptr, n, m, P, &L);
}

extern "C" hef_status hef_build_incidence(int64_t n, int64_t m, int64_t P, const int64_t* eptr,
                                          const int32_t* pins, const double* w,
                                          int32_t clique_mode, void* workspace,
                                          size_t workspace_bytes, void* stream,
                                          hef_incidence** out) {
  HEF_NVTX("hef_build_incidence (Algorithm 1 steps 1-2)");
  if (!out) return set_error(HEF_ERR_INVALID_ARG, "hef_build_incidence: out is NULL");
  *out = nullptr;
  if (n < 1 || m < 0 || P < 0)
    return set_error(HEF_ERR_INVALID_ARG, "hef_build_incidence: need n >= 1, m >= 0, P >= 0");
  if (n >= (1ll << 31) - 1 || m >= (1ll << 31) - 1 || P >= (1ll << 31) - 1)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_build_incidence: n, m and P must be < 2^31 - 1");
  if (!eptr || (P > 0 && !pins) || (m > 0 && !w))
    return set_error(HEF_ERR_INVALID_ARG, "hef_build_incidence: NULL input array");
  if (clique_mode != HEF_CLIQUE_HYPEREDGE && clique_mode != HEF_CLIQUE_PAPER)
    return set_error(HEF_ERR_INVALID_ARG, "hef_build_incidence: unknown clique_mode %d", clique_mode);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return set_error(HEF_ERR_WORKSPACE, "hef_build_incidence: workspace NULL or not 256-byte aligned");
  IncLayout L;
  size_t need = carve_incidence(workspace, n, m, P, &L);
  if (workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_build_incidence: workspace %zu bytes < %zu needed",
                     workspace_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hef_incidence* h = static_cast<hef_incidence*>(malloc(sizeof(hef_incidence)));
  if (!h) return set_error(HEF_ERR_INVALID_ARG, "hef_build_incidence: host malloc failed");
  *h = L.h;
  h->n = n;
  h->m = m;
  h->P = P;
  h->clique_mode = clique_mode;

  auto fail = [&](hef_status s) {
    free(h);
    return s;
  };
#define HEF_TRY(x)                 \
  do {                             \
    hef_status s_ = (x);           \
    if (s_ != HEF_OK) return fail(s_); \
  } while (0)
#define HEF_TRY_CUDA(call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(set_error(HEF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_))); \
  } while (0)

  HEF_TRY_CUDA(cudaMemsetAsync(h->status, 0, 64 * sizeof(unsigned int), st));
  HEF_TRY_CUDA(cudaMemsetAsync(h->status + 1, 0xFF, sizeof(unsigned int), st));
  HEF_TRY_CUDA(cudaMemsetAsync(L.tmp, 0, sizeof(int) * ((m > n ? m : n) + 1), st));

  // 1. validation and locality keys (one thread per hyperedge)
  {
    int grid = stride_grid(m > 0 ? m : 1, 8);
    HEF_LAUNCH("k_validate", st, k_validate<<<grid, kThreads, 0, st>>>((int)n, (int)m, P, eptr, pins, w,
                                                                       h->status, L.keys, L.vals, L.tmp));
    HEF_TRY_CUDA(cudaGetLastError());
  }
  // 2. locality schedule of hyperedges: stable counting sort by smallest pin
  // (bucket offsets in vptr, which the transpose fills later)
  if (m > 0) {
    int grid = stride_grid(m);
    HEF_TRY(exclusive_scan(L.tmp, h->vptr, n, L.scan_bsum, L.sb.counter, st, h->status));
    HEF_TRY_CUDA(cudaMemsetAsync(L.cur, 0, sizeof(int) * (n + 1), st));
    HEF_LAUNCH("k_place", st, k_place<<<grid, kThreads, 0, st>>>(m, reinterpret_cast<const int32_t*>(L.keys),
                                                                h->vptr, L.cur, h->status, L.place));
    HEF_TRY_CUDA(cudaGetLastError());
    HEF_LAUNCH("k_bucket_order", st, k_bucket_order<<<stride_grid(n), kThreads, 0, st>>>(
                                         n, h->vptr, L.place, nullptr, h->status, L.vals, nullptr));
    HEF_TRY_CUDA(cudaGetLastError());
    // internal CSC offsets
    HEF_LAUNCH("k_edge_sizes", st, k_edge_sizes<<<grid, kThreads, 0, st>>>((int)m, eptr, L.vals, h->status, L.tmp));
    HEF_TRY_CUDA(cudaGetLastError());
    HEF_TRY(exclusive_scan(L.tmp, h->ceptr, m, L.scan_bsum, L.sb.counter, st, h->status));
    HEF_TRY_CUDA(cudaMemsetAsync(L.tmp, 0, sizeof(int) * (n + 1), st));
    HEF_LAUNCH("k_edge_fill", st, k_edge_fill<<<grid, kThreads, 0, st>>>((int)m, clique_mode, eptr, pins, w, L.vals, h->ceptr,
                                           h->status, h->counter, h->perm, h->cpins, h->slot_edge,
                                           h->ew, h->ewh, h->ez, h->f_ew, h->f_ewh, h->f_ez, L.ec, L.tmp,
                                           L.part, h->totals));
    HEF_TRY_CUDA(cudaGetLastError());
    // list of large hyperedges (scored by whole CTAs)
    HEF_LAUNCH("k_big_flags", st, k_big_flags<<<grid, kThreads, 0, st>>>((int)m, h->ceptr, h->status,
                                                                        h->big_pos));
    HEF_TRY_CUDA(cudaGetLastError());
    HEF_TRY(exclusive_scan(h->big_pos, h->big_pos, m, L.scan_bsum, L.sb.counter, st, h->status));
    HEF_LAUNCH("k_windows", st, k_windows<<<stride_grid(m + 1), kThreads, 0, st>>>(
                                    (int)m, P, h->ceptr, h->status, h->win_edge));
    HEF_TRY_CUDA(cudaGetLastError());
    HEF_LAUNCH("k_big_scatter", st, k_big_scatter<<<grid, kThreads, 0, st>>>(
                                        (int)m, h->ceptr, h->big_pos, h->status, h->big_idx));
    HEF_TRY_CUDA(cudaGetLastError());
  } else {
    HEF_TRY_CUDA(cudaMemsetAsync(h->ceptr, 0, sizeof(int32_t), st));
    HEF_TRY_CUDA(cudaMemsetAsync(h->big_pos, 0, sizeof(int32_t), st));
    HEF_TRY_CUDA(cudaMemsetAsync(h->win_edge, 0, sizeof(int32_t) * (num_windows(P) + 1), st));
    HEF_TRY_CUDA(cudaMemsetAsync(h->totals, 0, 8 * sizeof(double), st));
  }
  // 3. vertex-major transpose: stable counting sort of the CSC slots by
  // vertex (the degree counts of k_edge_fill, scanned, are the offsets)
  HEF_TRY(exclusive_scan(L.tmp, h->vptr, n, L.scan_bsum, L.sb.counter, st, h->status));
  if (P > 0) {
    int grid = stride_grid(P);
    HEF_TRY_CUDA(cudaMemsetAsync(L.cur, 0, sizeof(int) * (n + 1), st));
    HEF_LAUNCH("k_place", st, k_place<<<grid, kThreads, 0, st>>>(P, h->cpins, h->vptr, L.cur, h->status,
                                                                L.place));
    HEF_TRY_CUDA(cudaGetLastError());
    HEF_LAUNCH("k_bucket_order", st, k_bucket_order<<<stride_grid(n), kThreads, 0, st>>>(
                                         n, h->vptr, L.place, h->slot_edge, h->status, h->vslot, h->vedge));
    HEF_TRY_CUDA(cudaGetLastError());
  }
  // 4. vertex degrees of both expansions and their totals
  {
    int grid = stride_grid(n);
    HEF_LAUNCH("k_node_scalars", st, k_node_scalars<<<grid, kThreads, 0, st>>>((int)n, h->vptr, h->vedge, L.ec, h->ewh, h->ez,
                                              h->status, h->counter, h->dc, h->db, h->inv_dc,
                                              h->inv_db, h->wsc, h->f_dc, h->f_db, h->f_inv_dc,
                                              h->f_inv_db, h->f_wsc, L.part, h->totals));
    HEF_TRY_CUDA(cudaGetLastError());
  }
#undef HEF_TRY
#undef HEF_TRY_CUDA
  *out = h;
  return HEF_OK;
}

extern "C" hef_status hef_incidence_check(const hef_incidence* inc, void* stream, uint32_t* detail,
                                          int64_t* where) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "hef_incidence_check: NULL handle");
  unsigned int st_host[2] = {0, 0};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HEF_CHECK_CUDA(cudaMemcpyAsync(st_host, inc->status, sizeof(st_host), cudaMemcpyDeviceToHost, st));
  HEF_CHECK_CUDA(cudaStreamSynchronize(st));
  if (detail) *detail = st_host[0];
  if (where) *where = st_host[0] ? (int64_t)st_host[1] : -1;
  if (st_host[0] & HEF_WAIT_TIMEOUT)
    return set_error(HEF_ERR_TIMEOUT, "a bounded grid-wide wait of the Krylov launch expired");
  if (st_host[0] & HEF_BOUNDS)
    return set_error(HEF_ERR_BOUNDS, "a kernel read an incidence index outside its array (bits 0x%x)",
                     st_host[0]);
  if (st_host[0])
    return set_error(HEF_ERR_INVALID_INPUT,
                     "hypergraph rejected by device validation (bits 0x%x, hyperedge %u)",
                     st_host[0], st_host[1]);
  return HEF_OK;
}

extern "C" hef_status hef_debug_set_pin(const hef_incidence* inc, int64_t slot, int32_t value,
                                        void* stream) {
  if (!HEF_DEBUG)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_debug_set_pin: only in the bounds-checked build");
  if (!inc || slot < 0 || slot >= inc->P)
    return set_error(HEF_ERR_INVALID_ARG, "hef_debug_set_pin: NULL handle or slot outside [0, P)");
  // a pinned staging word per call would outlive the asynchronous copy only
  // with a synchronisation; the copy is small, so it is made synchronous
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HEF_CHECK_CUDA(cudaMemcpyAsync(const_cast<int32_t*>(inc->cpins) + slot, &value, sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st));
  HEF_CHECK_CUDA(cudaStreamSynchronize(st));
  return HEF_OK;
}

extern "C" hef_status hef_incidence_sizes(const hef_incidence* inc, int64_t* n, int64_t* m,
                                          int64_t* P) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "hef_incidence_sizes: NULL handle");
  if (n) *n = inc->n;
  if (m) *m = inc->m;
  if (P) *P = inc->P;
  return HEF_OK;
}

extern "C" void hef_free_incidence(hef_incidence* inc) { free(inc); }

extern "C" hef_status hef_incidence_export(const hef_incidence* inc, int32_t* perm, int32_t* vptr,
                                           int32_t* vedge, double* dc, double* db, void* stream) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "hef_incidence_export: NULL handle");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (perm && inc->m > 0)
    HEF_CHECK_CUDA(cudaMemcpyAsync(perm, inc->perm, inc->m * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (vptr)
    HEF_CHECK_CUDA(cudaMemcpyAsync(vptr, inc->vptr, (inc->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (vedge && inc->P > 0) {
    HEF_LAUNCH("k_export_vedge", st, k_export_vedge<<<stride_grid(inc->P), kThreads, 0, st>>>(inc->P, inc->vedge, inc->perm, vedge));
    HEF_CHECK_LAUNCH();
  }
  if (dc) HEF_CHECK_CUDA(cudaMemcpyAsync(dc, inc->dc, inc->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (db) HEF_CHECK_CUDA(cudaMemcpyAsync(db, inc->db, inc->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return HEF_OK;
}
