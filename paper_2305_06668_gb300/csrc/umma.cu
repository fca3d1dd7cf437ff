// FP32 Gram matrices C = A^T B (the projected matrices of Algorithm 1 and the overlaps of
// Eq. (CDOrtho) in the FP32 phase of the mixed form) on the 5th-generation tensor cores.
//
// One persistent CTA per SM streams a contiguous range of rows in chunks of KC rows through
// a warp-specialised pipeline (448 threads):
//   * warp 0, one thread: the producer.  Each distinct row-major block behind A and B (a
//     block used by both, as in W^T W, is copied once) is one contiguous range per chunk:
//     one 1-D TMA bulk copy each into a ring of raw stages, completing on the stage's
//     mbarrier with the byte count;
//   * warps 6..13: the splitters, in one group or two groups of four that take the chunks
//     in turn (so one group's hand-offs overlap the other's work).  Each lane takes one
//     column and eight consecutive rows of a landed chunk and writes the TF32 parts
//     hi = rna(x) and lo = x - hi (exact; the tensor core reads its leading bits) as two
//     16-byte rows of core matrices (8 columns x 16 bytes) in the K-major no-swizzle layout
//     of the MMA, so a warp fills four core matrices with conflict-free 128-byte stores.
//     A warp's (column, row-group) units and their offsets are fixed for the whole launch
//     and computed once.  When A and B are the same block only A is split and the MMA
//     reads A's tiles for B;
//   * warp 1, one thread: the MMA issuer (tcgen05.mma kind::tf32, FP32 accumulation in
//     TMEM).  Operands of at most 64 columns are stacked: rows 0..63 of the A operand hold
//     A hi, rows 64..127 A lo, likewise the 128 columns of the B operand, so ONE M = 128,
//     N = 128 MMA per 8-row K step forms hi*hi and hi*lo (lanes 0..63) and lo*hi (lanes
//     64..127) in separate accumulator quadrants; wider operands take three MMAs per K step
//     (lo*hi, hi*lo, hi*hi) into one accumulator.  About 21 bits per product either way:
//     FP32-level accuracy.  tcgen05.commit releases the chunk's tiles and hands the
//     accumulator to the epilogue;
//   * warps 2..5: the epilogue.  Each warp reads its 32 TMEM lanes of the chunk's
//     accumulator (tcgen05.ld) and adds them to FP32 running sums with round-to-nearest
//     adds, so the tensor core's own accumulation never spans more than one chunk (carried
//     over thousands of rows its rounding would bias the sums).  The lo*hi sums of lanes
//     64..127 meet the hi*hi + hi*lo sums of lanes 0..63 once, at the end.
// Raw stages, tile buffers and accumulators each cycle through full / empty mbarriers, so
// copies, splits, MMAs and the epilogue of different chunks overlap.  The per-CTA sums go
// out in FP64 and are reduced in a fixed order by the caller.  Every wait is bounded: a
// thread that gives up sets a flag that makes every other wait return, the copies and
// MMAs in flight are waited for (bounded), TMEM is freed and the kernel returns.
#include <algorithm>

#include "common.cuh"
#include "umma.cuh"

namespace lobpcg {
namespace {

using namespace umma;

constexpr int kUM = 128;        // MMA M: columns of A (zero-padded), or A hi over A lo
constexpr int kMaxTS = 4;       // tile buffers (split -> MMA), chosen at launch
constexpr int kAS = 2;          // TMEM accumulators (MMA -> epilogue)
constexpr int kMaxRS = 6;       // raw ring stages (copy -> split), chosen at launch
constexpr int kMaxU = 6;        // distinct row-major blocks behind A and B
constexpr int kSplit0 = 6;      // first splitter warp
constexpr int kSplitWarps = 8;  // warps 6..13
constexpr int kThreads = 32 * (kSplit0 + kSplitWarps);
constexpr uint32_t kLBO = 128;  // bytes between core matrices along K
constexpr long long kWaitCycles = 1ll << 31;  // ~1 s at the SM clock: a wait that long has failed
constexpr size_t kSmemBudget = 220 * 1024;

__host__ __device__ constexpr uint32_t tmem_cols(int cols) {
  return cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}

// Set by a CTA that gave up waiting (1: a bulk copy, 2: an MMA, 3: a pipeline stage).
// Device code names it directly; the host reads it with cudaMemcpyFromSymbol (its
// host-side name is not a device address and is never passed to a kernel).
__device__ int g_umma_err = 0;

// x rounded to TF32 (10 stored mantissa bits), to nearest with ties away from zero: half a
// unit of the 13 dropped bits is added to the magnitude bits, then they are cleared (a
// carry into the exponent is the correct rounding up).  Finite x only.
__device__ __forceinline__ uint32_t to_tf32(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }

// Wait bounded in time (kWaitCycles) that also returns (false) once another thread of the
// CTA gave up.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int code) {
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 15u) == 15u) {
      if (*abort_flag) return false;
      if (clock64() - t0 > kWaitCycles) break;
    }
  }
  *abort_flag = 1;
  atomicExch(&g_umma_err, code);
  return false;
}

// STACK: both operands at most 64 columns, one stacked MMA per K step; otherwise three.
template <int NP, int KC, bool STACK>
__global__ void __launch_bounds__(kThreads, 1) gram_umma_kernel(int64_t n, Cols<float> A, Cols<float> B, int ld,
                                                                int upper, int rs, int ts, int groups,
                                                                double* __restrict__ part,
                                                                int64_t rows_per_cta) {
  constexpr int N = 16 * NP;             // columns of C per running sum (>= pb)
  constexpr int MN = STACK ? 128 : N;    // MMA N, and TMEM columns of one accumulator
  constexpr uint32_t kSBO = 32 * KC;     // bytes between core matrices along M / N
  // units per splitter warp: (2 + 2) column groups x 4 row groups / 4 warps (stacked, two
  // splitter groups) or (3 + 3) x 8 / 8 (one group)
  constexpr int kMaxUW = STACK ? 8 : 6;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t raw_full[kMaxRS], raw_empty[kMaxRS], tile_full[kMaxTS], tile_empty[kMaxTS];
  __shared__ uint64_t acc_full[kAS], acc_empty[kAS];
  __shared__ const float* useg[kMaxU];
  __shared__ int ucopy[kMaxU];      // floats of the last row each block's copy needs
  __shared__ int colofs[2][kMaxS];  // column -> float offset in a raw stage (-1: none)
  __shared__ int nu_s, same_s;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int pa = A.width(), pb = B.width();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int seg_floats = KC * ld;

  if (tid == 0) {
    int nu = 0;
    for (int o = 0; o < 2; ++o) {
      const Cols<float>& c = o == 0 ? A : B;
      for (int g = 0; g < c.nseg; ++g) {
        int u = 0;
        while (u < nu && useg[u] != c.p[g]) ++u;
        if (u == nu) useg[nu] = c.p[g], ucopy[nu] = 0, ++nu;
        ucopy[u] = max(ucopy[u], (c.w[g] + 3) / 4 * 4);
      }
    }
    bool same = A.nseg == B.nseg;
    for (int g = 0; same && g < A.nseg; ++g) same = A.p[g] == B.p[g] && A.w[g] == B.w[g];
    nu_s = nu, same_s = same ? 1 : 0;
    abort_flag = 0;
    const int wpg = kSplitWarps / groups;  // splitter warps per chunk
    for (int s = 0; s < kMaxRS; ++s) mbar_init(&raw_full[s], 1), mbar_init(&raw_empty[s], wpg);
    for (int s = 0; s < kMaxTS; ++s) mbar_init(&tile_full[s], wpg), mbar_init(&tile_empty[s], 1);
    for (int s = 0; s < kAS; ++s) mbar_init(&acc_full[s], 1), mbar_init(&acc_empty[s], 4);
    fence_barrier_init();
  }
  __syncthreads();
  const int nu = nu_s;
  const bool same = same_s != 0;
  for (int i = tid; i < 2 * kMaxS; i += blockDim.x) {
    const int o = i / kMaxS, m = i % kMaxS;
    const Cols<float>& c = o == 0 ? A : B;
    int off = -1;
    if (m < c.width()) {
      int base = 0, g = 0;
      while (m >= base + c.w[g]) base += c.w[g], ++g;
      int u = 0;
      while (useg[u] != c.p[g]) ++u;
      off = u * seg_floats + (m - base);
    }
    colofs[o][m] = off;
  }

  // tiles, per buffer: A hi, A lo, B hi, B lo (B's absent when B is A).  Stacked: 8
  // core-matrix rows (64 columns, zero-padded) each, so A lo continues A hi as rows
  // 64..127 of the M = 128 operand, likewise B.  Otherwise A has GA = ceil(pa / 8) rows and
  // B N / 8; an M = 128 MMA then reads 16 core-matrix rows of A from its base, past A's GA
  // rows into the following tiles (or the pad after the last buffer), which only feeds
  // accumulator lanes >= pa, never read; likewise B's rows >= pb.
  const int GA = STACK ? 8 : (pa + 7) / 8;
  const int TA = GA * (int)kSBO / 4;                                           // words
  const int TB = same ? 0 : STACK ? 8 * (int)kSBO / 4 : N * KC;                // words
  // the raw ring; it also holds the stacked epilogue's final exchange (64 x N floats)
  const size_t raw_bytes = max(((size_t)rs * nu * seg_floats * 4 + 127) / 128 * 128, STACK ? (size_t)64 * N * 4 : 0);
  float* raw = reinterpret_cast<float*>(smem);  // [rs][nu][KC][ld]
  uint32_t* tiles = reinterpret_cast<uint32_t*>(smem + raw_bytes);
  const int tbuf = 2 * TA + 2 * TB;  // words of one tile buffer
  // zero the tiles and the pad (columns past pa / pb are never written)
  const int pad = STACK ? 0 : max(0, kUM / 8 * (int)kSBO / 4 - TA - 2 * TB);
  for (int e = tid; e < ts * tbuf + pad; e += blockDim.x) tiles[e] = 0u;
  __syncwarp();
  if (warp == 1) tmem_alloc(&tmem_slot, tmem_cols(kAS * MN));
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + KC - 1) / KC) : 0;
  int issued = 0, committed = 0;  // producer / MMA thread only
  if (warp == 0) {
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;  // ring slot of chunk c and the parity of its round (c / rs)
      for (int c = 0; c < nchunks; ++c) {
        if (c >= rs && !wait_bar(&raw_empty[st], ph ^ 1u, &abort_flag, 3)) break;
        const int64_t r0 = r_begin + (int64_t)c * KC;
        const int rows = (int)min((int64_t)KC, r_end - r0);
        // every row in full (ld floats) but the last, of which only the used columns
        // (rounded up to 16 bytes): the copy never reads past the block's last element
        uint32_t total = 0;
        for (int u = 0; u < nu; ++u) total += (uint32_t)((rows - 1) * ld + ucopy[u]) * 4u;
        mbar_expect_tx(&raw_full[st], total);
        for (int u = 0; u < nu; ++u)
          bulk_g2s(raw + ((size_t)st * nu + u) * seg_floats, useg[u] + r0 * ld,
                   (uint32_t)((rows - 1) * ld + ucopy[u]) * 4u, &raw_full[st]);
        issued = c + 1;
        if (++st == rs) st = 0, ph ^= 1u;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kUM, MN);
      // descriptors of tile buffer 0; buffer b and K step kk add b * tbuf words and kk *
      // 256 bytes to the start address (encoded >> 4; every address stays below 256 KB)
      const uint32_t t0 = smem_addr(tiles);
      const uint32_t oAl = (uint32_t)TA * 4u, oB = same ? 0u : 2u * TA * 4u,
                     oBl = same ? oAl : (uint32_t)(2 * TA + TB) * 4u;
      const uint64_t dA = desc_kmajor(t0, kLBO, kSBO), dAl = desc_kmajor(t0 + oAl, kLBO, kSBO);
      const uint64_t dB = desc_kmajor(t0 + oB, kLBO, kSBO), dBl = desc_kmajor(t0 + oBl, kLBO, kSBO);
      int buf = 0, r = 0;
      uint32_t tph = 0, aph = 0;  // tile / accumulator slots and round parities
      for (int c = 0; c < nchunks; ++c) {
        if (!wait_bar(&tile_full[buf], tph, &abort_flag, 3)) break;
        if (c >= kAS && !wait_bar(&acc_empty[r], aph ^ 1u, &abort_flag, 3)) break;
        tc_fence_after();
        const uint64_t bo = (uint64_t)((uint32_t)(buf * tbuf * 4) >> 4);
        const uint32_t d = tmem + (uint32_t)(r * MN);
#pragma unroll
        for (int kk = 0; kk < KC / 8; ++kk) {
          const uint64_t ko = bo + (uint64_t)(kk * 16);  // kk * 2 * kLBO bytes
          if constexpr (STACK) {
            mma_tf32(d, dA + ko, dB + ko, idesc, kk);
          } else {
            mma_tf32(d, dAl + ko, dB + ko, idesc, kk);
            mma_tf32(d, dA + ko, dBl + ko, idesc, 1);
            mma_tf32(d, dA + ko, dB + ko, idesc, 1);
          }
        }
        mma_commit(&tile_empty[buf]);
        mma_commit(&acc_full[r]);
        committed = c + 1;
        if (++buf == ts) buf = 0, tph ^= 1u;
        if (++r == kAS) r = 0, aph ^= 1u;
      }
    }
  } else if (warp < kSplit0) {
    // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31
    const int quad = warp & 3;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    float acc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = 0.f;
    int r = 0, c = 0;
    uint32_t aph = 0;
    for (; c < nchunks; ++c) {
      if (!__all_sync(0xffffffffu, wait_bar(&acc_full[r], aph, &abort_flag, 2))) break;
      tc_fence_after();
      const uint32_t a0 = tmem + lane_base + (uint32_t)(r * MN);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        float v[16];
        tmem_ld16(a0 + 16 * q, v);
        if (STACK && quad < 2) {  // hi*hi + hi*lo
          float w[16];
          tmem_ld16(a0 + 64 + 16 * q, w);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = __fadd_rn(v[i], w[i]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[16 * q + i] = __fadd_rn(acc[16 * q + i], v[i]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[r]);
      if (++r == kAS) r = 0, aph ^= 1u;
    }
    // every chunk's MMAs done means every copy landed: the raw ring is idle
    const bool done = c == nchunks;
    double* out = part + (int64_t)blockIdx.x * pa * pb;
    const int row = 32 * quad + lane;
    if (STACK) {
      // lanes 64..127 (lo*hi) hand their sums to lanes 0..63 through the raw ring
      float* red = reinterpret_cast<float*>(smem);
      if (quad >= 2 && done)
#pragma unroll
        for (int j = 0; j < N; ++j) red[j * 64 + row - 64] = acc[j];
      asm volatile("bar.sync 3, 128;\n" ::: "memory");  // the four epilogue warps
      if (quad < 2 && row < pa) {
        const bool ok = done && !abort_flag;
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (j < pb && (!upper || row <= j))
            out[row + (int64_t)j * pa] = ok ? (double)__fadd_rn(acc[j], red[j * 64 + row]) : 0.0;
      }
    } else if (row < pa) {
      const bool ok = done && !abort_flag;
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (j < pb && (!upper || row <= j)) out[row + (int64_t)j * pa] = ok ? (double)acc[j] : 0.0;
    }
  } else {
    // The splitter warps form `groups` groups that take the chunks in turn (group g: chunks
    // g, g + groups, ..), so the hand-offs of one chunk overlap the splits of the next.  The
    // units (32 columns x 8 rows of one operand) of a warp are the same in every chunk: unit
    // u = sg + j * wpg.  Per unit the lane's source offset in a raw stage and its
    // destination word in a tile buffer are computed once.
    const int wpg = kSplitWarps / groups;
    const int sw = warp - kSplit0, g = sw / wpg, sg = sw % wpg;
    const int gA = (pa + 31) / 32, gB = same ? 0 : (pb + 31) / 32;
    constexpr int K8 = KC / 8;  // 8-row groups per chunk
    const int units = (gA + gB) * K8;
    const int my = units > sg ? (units - sg + wpg - 1) / wpg : 0;  // <= kMaxUW
    int src[kMaxUW];       // float offset in a raw stage of the unit's first row (-1: none)
    uint32_t dst[kMaxUW];  // word in a tile buffer | isA << 20 | k8 << 21
#pragma unroll
    for (int j = 0; j < kMaxUW; ++j) {
      const int u = sg + j * wpg;
      src[j] = -1, dst[j] = 0;
      if (j < my) {
        const bool isA = u < gA * K8;
        const int v = isA ? u : u - gA * K8;
        const int grp = v / K8, k8 = v % K8;
        const int m = grp * 32 + lane;
        const int off = colofs[isA ? 0 : 1][m];
        if (off >= 0) {
          src[j] = off + 8 * k8 * ld;
          // core-matrix rows 2 k8 and 2 k8 + 1 along K of column m
          const uint32_t w = (isA ? 0u : 2u * TA) + (((uint32_t)(m >> 3) * kSBO + (uint32_t)(2 * k8) * kLBO) >> 2) +
                             4u * (m & 7);
          dst[j] = w | (isA ? 1u << 20 : 0u) | (uint32_t)k8 << 21;
        }
      }
    }
    // hi = rna(x) to TF32; lo = x - hi exactly (the tensor core reads lo's leading 11 bits)
    auto split = [&](const float (&x)[8], uint32_t* th, uint32_t* tl) {
      uint32_t h[8], l[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        h[i] = to_tf32(x[i]);
        l[i] = __float_as_uint(__fsub_rn(x[i], __uint_as_float(h[i])));
      }
      *reinterpret_cast<uint4*>(th) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(th + kLBO / 4) = make_uint4(h[4], h[5], h[6], h[7]);
      *reinterpret_cast<uint4*>(tl) = make_uint4(l[0], l[1], l[2], l[3]);
      *reinterpret_cast<uint4*>(tl + kLBO / 4) = make_uint4(l[4], l[5], l[6], l[7]);
    };
    int st = g % rs, buf = g % ts;
    uint32_t ph = 0, tph = 0;
    for (int c = g; c < nchunks; c += groups) {
      if (!__all_sync(0xffffffffu, wait_bar(&raw_full[st], ph, &abort_flag, 1))) break;
      if (c >= ts && !__all_sync(0xffffffffu, wait_bar(&tile_empty[buf], tph ^ 1u, &abort_flag, 2))) break;
      const int rows = (int)min((int64_t)KC, r_end - (r_begin + (int64_t)c * KC));
      const float* rsb = raw + (size_t)st * nu * seg_floats;
      uint32_t* tb = tiles + buf * tbuf;
      if (rows == KC) {
        // two units per pass: their 16 loads are in flight together
#pragma unroll
        for (int j0 = 0; j0 < kMaxUW; j0 += 2) {
          if (j0 < my) {
            float x[2][8];
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
              for (int i = 0; i < 8; ++i) x[e][i] = src[j0 + e] >= 0 ? rsb[src[j0 + e] + i * ld] : 0.f;
#pragma unroll
            for (int e = 0; e < 2; ++e)
              if (src[j0 + e] >= 0) {
                uint32_t* th = tb + (dst[j0 + e] & 0xfffffu);
                split(x[e], th, th + ((dst[j0 + e] >> 20) & 1u ? TA : TB));
              }
          }
        }
      } else {
        // the last chunk of the CTA's range: rows past its end read as zero
#pragma unroll
        for (int j = 0; j < kMaxUW; ++j) {
          if (j >= my || src[j] < 0) continue;
          const int k0 = 8 * (int)(dst[j] >> 21);
          float x[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) x[i] = k0 + i < rows ? rsb[src[j] + i * ld] : 0.f;
          uint32_t* th = tb + (dst[j] & 0xfffffu);
          split(x, th, th + ((dst[j] >> 20) & 1u ? TA : TB));
        }
      }
      // the split tiles go to the tensor core (async proxy); the MMA thread waits for
      // every warp of the group
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&raw_empty[st]);
        mbar_arrive(&tile_full[buf]);
      }
      if ((st += groups) >= rs) st -= rs, ph ^= 1u;
      if ((buf += groups) >= ts) buf -= ts, tph ^= 1u;
    }
  }
  __syncthreads();
  if (abort_flag) {
    // give the copies and MMAs this CTA issued a bounded chance to complete before its
    // shared memory and tensor memory go
    if (warp == 0 && lane == 0)
      for (int c = max(0, issued - rs); c < issued; ++c) mbar_wait(&raw_full[c % rs], (uint32_t)(c / rs) & 1u, kWaitCycles);
    if (warp == 1 && lane == 0 && committed > 0)
      mbar_wait(&acc_full[(committed - 1) % kAS], (uint32_t)((committed - 1) / kAS) & 1u, kWaitCycles);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols(kAS * MN));
  }
}

__global__ void umma_err_reset_kernel() { g_umma_err = 0; }

// Launch plan: rows per chunk, raw stages, dynamic shared memory.
struct UmmaPlan {
  int kc = 0, rs = 0, ts = 0, groups = 1, nu = 0;
  bool same = false, stack = false;
  size_t smem = 0;
};

bool umma_plan(const Cols<float>& a, const Cols<float>& b, int ld, UmmaPlan& pl) {
  const float* u[kMaxU];
  int nu = 0;
  for (int o = 0; o < 2; ++o) {
    const Cols<float>& c = o == 0 ? a : b;
    for (int g = 0; g < c.nseg; ++g) {
      int i = 0;
      while (i < nu && u[i] != c.p[g]) ++i;
      if (i == nu) u[nu++] = c.p[g];
    }
  }
  bool same = a.nseg == b.nseg;
  for (int g = 0; same && g < a.nseg; ++g) same = a.p[g] == b.p[g] && a.w[g] == b.w[g];
  const int pa = a.width(), pb = b.width(), N = (pb + 15) / 16 * 16;
  const bool stack = pa <= 64 && pb <= 64;
  // thin operands take 64-row chunks (fewer pipeline hand-offs per byte), wide ones 32
  const int kc = (size_t)32 * nu * ld * 4 < 8 * 1024 ? 64 : 32;
  const size_t sbo = 32 * (size_t)kc;
  const size_t ta = (stack ? 8 : (size_t)(pa + 7) / 8) * sbo;
  const size_t tb = same ? 0 : stack ? 8 * sbo : (size_t)N * kc * 4;
  // unstacked: the M = 128 read of the last buffer's A lo tile (16 core-matrix rows) stays inside
  const size_t reach = (size_t)kUM / 8 * sbo, after = ta + 2 * tb;
  const size_t pad = !stack && reach > after ? reach - after : 0;
  const size_t stage = (size_t)kc * nu * ld * 4;
  // as many tile buffers as leave room for as many raw stages (at least two of each)
  int ts = kMaxTS;
  while (ts > 2 && ts * (2 * ta + 2 * tb) + pad + ts * stage + 128 > kSmemBudget) --ts;
  const size_t fixed = ts * (2 * ta + 2 * tb) + pad;
  if (fixed + 2 * stage + 128 > kSmemBudget) return false;
  const int rs = (int)std::min<size_t>(kMaxRS, (kSmemBudget - fixed - 128) / stage);
  pl.kc = kc, pl.rs = rs, pl.ts = ts, pl.nu = nu, pl.same = same, pl.stack = stack;
  // two splitter groups when the rings hold two chunks being split besides the MMA's
  pl.groups = stack && ts >= 4 && rs >= 4 ? 2 : 1;
  // the raw ring also holds the stacked epilogue's final exchange (64 x N floats)
  pl.smem = std::max((rs * stage + 127) / 128 * 128, stack ? (size_t)64 * N * 4 : 0) + fixed;
  if (pl.smem > kSmemBudget) return false;
  return true;
}

template <int NP, int KC, bool STACK>
int umma_launch(int64_t n, const Cols<float>& a, const Cols<float>& b, int ld, bool upper, double* part, int max_ctas,
                const UmmaPlan& pl, cudaStream_t st) {
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(gram_umma_kernel<NP, KC, STACK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBudget));
    return true;
  }();
  (void)attr;
  // one CTA per SM (one wave; each streams a contiguous range of rows)
  int dev = 0, sms = 152;
  LB_CUDA(cudaGetDevice(&dev));
  LB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int64_t ctas = std::min<int64_t>(std::min<int64_t>(max_ctas, sms), ceil_div(n, KC));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + KC - 1) / KC * KC;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  gram_umma_kernel<NP, KC, STACK>
      <<<(unsigned)ctas, kThreads, pl.smem, st>>>(n, a, b, ld, upper ? 1 : 0, pl.rs, pl.ts, pl.groups, part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

template <int NP>
int umma_launch_kc(int64_t n, const Cols<float>& a, const Cols<float>& b, int ld, bool upper, double* part,
                   int max_ctas, const UmmaPlan& pl, cudaStream_t st) {
  if constexpr (NP <= 4) {
    if (pl.stack)
      return pl.kc == 64 ? umma_launch<NP, 64, true>(n, a, b, ld, upper, part, max_ctas, pl, st)
                         : umma_launch<NP, 32, true>(n, a, b, ld, upper, part, max_ctas, pl, st);
  }
  return pl.kc == 64 ? umma_launch<NP, 64, false>(n, a, b, ld, upper, part, max_ctas, pl, st)
                     : umma_launch<NP, 32, false>(n, a, b, ld, upper, part, max_ctas, pl, st);
}

bool umma_aligned(const Cols<float>& c, int ld) {
  for (int g = 0; g < c.nseg; ++g)
    if (c.ld[g] != ld || c.w[g] > ld || (reinterpret_cast<uintptr_t>(c.p[g]) & 15)) return false;
  return true;
}

}  // namespace

// tcgen05 Gram partials (contract of gram_partials_pipe<float>); returns 0 without
// launching when the operands do not share one 16-byte aligned row stride (a multiple of
// 4 floats), are wider than 96 columns, or need more shared memory than a CTA has.
int gram_partials_umma(int64_t n, const Cols<float>& a, const Cols<float>& b, bool upper, double* part,
                       int max_ctas, cudaStream_t st) {
  if (a.nseg == 0 || b.nseg == 0 || n <= 0) return 0;
  const int ld = a.ld[0];
  if (ld % 4 != 0 || !umma_aligned(a, ld) || !umma_aligned(b, ld)) return 0;
  const int pa = a.width(), pb = b.width();
  if (pa > kMaxS || pb > kMaxS || pa < 1 || pb < 1) return 0;
  UmmaPlan pl;
  if (!umma_plan(a, b, ld, pl)) return 0;
  switch ((pb + 15) / 16) {
    case 1: return umma_launch_kc<1>(n, a, b, ld, upper, part, max_ctas, pl, st);
    case 2: return umma_launch_kc<2>(n, a, b, ld, upper, part, max_ctas, pl, st);
    case 3: return umma_launch_kc<3>(n, a, b, ld, upper, part, max_ctas, pl, st);
    case 4: return umma_launch_kc<4>(n, a, b, ld, upper, part, max_ctas, pl, st);
    case 5: return umma_launch_kc<5>(n, a, b, ld, upper, part, max_ctas, pl, st);
    default: return umma_launch_kc<6>(n, a, b, ld, upper, part, max_ctas, pl, st);
  }
}

// Reads and clears the give-up flag of the tcgen05 Gram (synchronises the stream); throws
// when a CTA gave up waiting, so the failure surfaces as ECUDA.
void umma_check(cudaStream_t st) {
  int flag = 0;
  LB_CUDA(cudaMemcpyFromSymbolAsync(&flag, g_umma_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  LB_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    umma_err_reset_kernel<<<1, 1, 0, st>>>();
    LB_LAUNCH_CHECK();
    LB_CUDA(cudaStreamSynchronize(st));
    throw CudaError(flag == 1   ? "tensor-core Gram: a bulk copy did not complete in time"
                    : flag == 2 ? "tensor-core Gram: an MMA did not complete in time"
                                : "tensor-core Gram: a pipeline stage was not released in time");
  }
}

}  // namespace lobpcg
