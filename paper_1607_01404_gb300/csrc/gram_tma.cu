// TMA-fed row Gram G = [P0 P1 P2]^T Q (the Table 3 inner products: the
// Rayleigh-Ritz projection V^T W and the Gram matrices of CGS and CholQR) for
// the F32 and DF64 storage modes, p <= 64 and q <= 8.
//
// Memory side: row tiles of every segment are streamed into a ring of shared-
// memory stages by the Tensor Memory Accelerator (cp.async.bulk.tensor.2d with
// an mbarrier per stage, one 2D tensor map per segment: rows x the segment's
// columns counted from the 16-byte boundary at or before its first column).
// Each stage has an mbarrier that completes when its copies have landed; the
// warps wait on it independently, and the last warp to finish a stage (an
// arrival counter in shared memory) refills it with the CTA's next chunk, so
// no CTA-wide barrier and no idle producer warp sit in the loop.  The bytes in
// flight cost no registers: a CTA keeps its ring's tiles in flight.
// Rows past r1 and columns past the segment are outside the tensor maps and
// arrive as zeros, so the ragged tail needs no masks.  Each of the TPR lanes
// of a row owns KP consecutive columns of a tile row (a segment's columns
// counted from its copy boundary, so a window that starts inside a 16-byte
// word brings a few columns before it, whose products are dropped) and reads
// them, and the row's Q columns, with 16- or 8-byte shared-memory loads; tile
// rows are padded so that the rows one load instruction touches start on
// distinct banks.
//
// Arithmetic side: FP64-class accumulation of every product of a lane's
// columns with the row's Q columns, and a fixed-order double-float reduction
// of the lanes (deterministic).
// * DF64 storage: Dot2 (Ogita, Rump and Oishi 2005): the exact product of the
//   hi parts (TwoProd by FMA) plus the cross terms, TwoSum into hi, rounding
//   errors into lo, renormalised every 2 rows (two Q columns per packed
//   f32x2 instruction where there are two or more); accurate to about 2^-48 of
//   the products, as the double-float data.
// * FP32 storage: anchored accumulation.  Pair (i, j) of a lane accumulates
//   into s = sigma_ij + partial sum, sigma_ij = a_i b_j a power of two of at
//   least 4 times the Cauchy-Schwarz bound sqrt(SP_i SQ_j) of the lane's
//   partial sums (SP, SQ: running sums of squares), so that
//       s' = fma(p, q, s),  z = s' - s  (exact: Sterbenz),  d = fma(p, q, -z)
//   is the rounding error of the update to FP32 precision, summed in c:
//   4 FP32 operations per product instead of Dot2's 10, issued as packed
//   f32x2 instructions for pairs of Q columns (2 instructions per product,
//   each half rounded as the scalar operation).  An outgrown anchor
//   is raised with 4x headroom and its pairs move to it by an error-free
//   FastTwoSum; every 8 rows c is folded into s.  The error of a product is
//   about 2^-47 sigma_ij, i.e. 2^-43 of the Cauchy-Schwarz bound of the
//   lane's rows: far below the 2^-24 of the FP32 data, but not the 2^-48 of
//   double-float data, which therefore keeps Dot2.  Entries must be below
//   2^50 in magnitude.
//
// Every mbarrier wait is bounded (about 2^31 SM cycles); a CTA whose wait
// runs out writes NaN partial sums, waits (bounded) for its copies in flight
// and returns, so the failure reaches the caller as a NaN Gram.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "f32x2.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace phsvds {

namespace {

using namespace tma;

constexpr int kT = 256;       // threads per CTA
constexpr int kMaxStages = 4;  // ring stages per CTA, at most
constexpr int kMaxSeg = 4;    // up to 3 P segments and Q
constexpr int kMaxP = 64;
constexpr int kMaxSmem = 200 * 1024 + 128;  // largest dynamic shared memory of a plan
constexpr int kBarBytes = kMaxStages * 8 + kMaxStages * 4 + 16;  // stage barriers, arrival counters, failure word
constexpr int kRingTwoCtas = 110 * 1024;         // a plan at most this large lets two CTAs share an SM

struct TmaSeg {
  int soff;    // float offset of the segment's tile inside a stage
  int bw;      // floats per tile row (box width)
  int pstart;  // first lane column of the segment (lane columns: see the kernel)
  int ncp;     // lane columns of the segment: xe + nc rounded up to KP
  int xe;      // elements before the segment's first column in its tile rows
  int nc;      // columns
  int c0;      // first column of the segment in P
};
struct TmaPlan {
  TmaSeg seg[kMaxSeg];  // [0, nP): P segments, [nP]: Q
  int nP;
  int stage_floats;  // a multiple of 32 (every tile starts on a 128-byte boundary)
  int R;             // rows per stage
  int stages;        // ring stages (2 .. kMaxStages)
  int bar_off;       // float offset of the stage barriers (after the ring and the reduction buffer)
};

// ---- anchored accumulation (see the file header) ----
__device__ __forceinline__ float hi_of(float x) { return x; }
__device__ __forceinline__ float hi_of(df x) { return x.hi; }
__device__ __forceinline__ float lo_of(df x) { return x.lo; }

__device__ __forceinline__ void anc_add(float& s, float& c, float x, float y) {
  const float t = s;
  s = __fmaf_rn(x, y, t);
  const float z = __fsub_rn(s, t);
  c = __fadd_rn(c, __fmaf_rn(x, y, -z));
}
// Dot2 step for double-float values: hi + lo += x y
__device__ __forceinline__ void dot2_add(float& hi, float& lo, df x, df y) {
  const df p = two_prod(x.hi, y.hi);
  const float pl = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  const df s = two_sum(hi, p.hi);
  hi = s.hi;
  lo = __fadd_rn(lo, __fadd_rn(s.lo, pl));
}
// smallest power of two a with a^2 >= 18 sp, at least 2^-58 (the floor keeps
// the bound valid for entries whose squares underflow)
__device__ __forceinline__ float anc_anchor(float sp) {
  const unsigned u = __float_as_uint(18.0f * sp);
  int e = (int)(u >> 23) - 127;
  if (u & 0x7fffffu) ++e;
  int ea = (e + 1) >> 1;
  ea = max(ea, -58);
  return __uint_as_float((unsigned)(ea + 127) << 23);
}
// moves pair (s, c) from anchor so to sn (|sn| >= 2 |so|): error-free
__device__ __forceinline__ void anc_move(float& s, float& c, float so, float sn) {
  const float v = __fsub_rn(s, so);
  const float t = __fadd_rn(sn, v);
  c = __fadd_rn(c, __fsub_rn(v, __fsub_rn(t, sn)));
  s = t;
}

// N consecutive floats from shared memory in the widest aligned pieces (the
// callers' offsets are multiples of the piece)
template <int N>
__device__ __forceinline__ void lds_n(const float* p, float (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 t = reinterpret_cast<const float4*>(p)[i];
      v[4 * i] = t.x;
      v[4 * i + 1] = t.y;
      v[4 * i + 2] = t.z;
      v[4 * i + 3] = t.w;
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 t = reinterpret_cast<const float2*>(p)[i];
      v[2 * i] = t.x;
      v[2 * i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}
template <class P>
__device__ __forceinline__ typename P::A elem(const float* v, int i);
template <>
__device__ __forceinline__ float elem<PF32>(const float* v, int i) {
  return v[i];
}
template <>
__device__ __forceinline__ df elem<PDF64>(const float* v, int i) {
  return df{v[2 * i], v[2 * i + 1]};
}

template <class P, int TPR, int KP, int NQ>
__global__ void __launch_bounds__(kT, 2)
    k_gram_tma(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
               const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap m3, const TmaPlan plan,
               long long r0, long long r1, int p, int q, df* __restrict__ partial) {
  using A = typename P::A;
  constexpr int E = P::id == kF32 ? 1 : 2;  // floats per element
  constexpr int RPC = kT / TPR;              // rows the CTA covers at once
  constexpr int NW = kT / 32;
  constexpr float kFloor = 3.4694470e-18f;   // 2^-58
  constexpr bool kAnchored = P::id == kF32;
  extern __shared__ __align__(128) float smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + plan.bar_off);
  int* arrived = reinterpret_cast<int*>(full + kMaxStages);
  int* fail = arrived + kMaxStages;
  const int NS = plan.stages;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = plan.R;
  const long long nchunks = (r1 - r0 + R - 1) / R;
  const int nseg = plan.nP + 1;
  unsigned tx_bytes = 0;
  for (int sg = 0; sg < nseg; ++sg) tx_bytes += (unsigned)(plan.seg[sg].bw * R * 4);
  // copies of chunk ch into stage st (one thread)
  auto issue = [&](long long ch, int st) {
    float* base = smem + (size_t)st * plan.stage_floats;
    mbar_expect_tx(&full[st], tx_bytes);
    const int y = (int)(r0 + ch * R);
    for (int sg = 0; sg < nseg; ++sg) {
      const CUtensorMap* m = sg == 0 ? &m0 : sg == 1 ? &m1 : sg == 2 ? &m2 : &m3;
      load_2d(base + plan.seg[sg].soff, m, 0, y, &full[st]);
    }
  };

  if (threadIdx.x == 0) {
    for (int st = 0; st < NS; ++st) {
      mbar_init(&full[st], 1);
      arrived[st] = 0;
    }
    *fail = 0;
    fence_mbar_init();
    for (int st = 0; st < NS; ++st) {
      const long long ch = blockIdx.x + (long long)st * gridDim.x;
      if (ch < nchunks) issue(ch, st);
    }
  }
  __syncthreads();

  // ---- the P columns of this lane ----
  // Lane columns: segment s occupies lane columns [pstart, pstart + ncp), in
  // the order of its tile rows: xe elements before its first column (the copy
  // starts on a 16-byte boundary), its nc columns, then zeros (the copies read
  // past the data) up to a multiple of KP.  Lane `part` owns the KP
  // consecutive lane columns from part KP, inside one segment, and reads them
  // with vector loads; lane columns past the last segment lie inside its
  // widened tile rows (zeros).  Products of the prefix and padding columns are
  // computed and dropped.
  const int part = threadIdx.x % TPR;
  const int pc0 = part * KP;
  int sgl = 0;
  while (sgl < plan.nP - 1 && pc0 >= plan.seg[sgl + 1].pstart) ++sgl;
  const int po = plan.seg[sgl].soff + (pc0 - plan.seg[sgl].pstart) * E;  // tile-row offset of the lane's columns
  const int pw = plan.seg[sgl].bw;
  const TmaSeg qs = plan.seg[plan.nP];
  // Q columns 0 .. NQ - 1 from the first column of Q (xe elements into its
  // tile rows): F32 reads them with 16/8-byte loads when that is a word
  // boundary, else one by one; double-float with 8-byte loads
  const int qo = qs.soff + qs.xe * E;
  const bool qvec = qs.xe == 0;

  float sa[KP][NQ], ca[KP][NQ];
  // two or more Q columns: the sums of Q columns 2h and 2h + 1 travel as one
  // register pair and update with packed instructions (the scalar updates'
  // roundings, half the instructions)
  constexpr bool kPack = NQ >= 2;
  constexpr int NH = NQ >= 2 ? NQ / 2 : 1;
  float2 s2[KP][NH], c2[KP][NH];
  const float2 neg1{-1.f, -1.f};
  // anchors a_k, b_j (powers of two), the running sums of squares and the
  // thresholds a^2 / 4.5 above which an anchor is raised
  float an[KP], bn[NQ], sp[KP], sq[NQ], ta[KP], tb[NQ];
  const float thr0 = kFloor * kFloor * (1.0f / 4.5f);
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    an[k] = kFloor;
    sp[k] = 0.f;
    ta[k] = thr0;
  }
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    bn[j] = kFloor;
    sq[j] = 0.f;
    tb[j] = thr0;
  }
#pragma unroll
  for (int k = 0; k < KP; ++k)
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      sa[k][j] = kAnchored ? kFloor * kFloor : 0.f;
      ca[k][j] = 0.f;
    }
#pragma unroll
  for (int k = 0; k < KP; ++k)
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      s2[k][h] = kAnchored ? float2{kFloor * kFloor, kFloor * kFloor} : float2{0.f, 0.f};
      c2[k][h] = float2{0.f, 0.f};
    }

  const int row0 = threadIdx.x / TPR;
  int it = 0, pairs = 0;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++it) {
    const int stage = it % NS;
    // warp-uniform decision: every lane of a warp leaves the loop together
    const bool ok =
        __all_sync(0xffffffffu, !*reinterpret_cast<volatile int*>(fail) && mbar_wait(&full[stage], (unsigned)((it / NS) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(fail, 1);
      break;
    }
    const float* tile = smem + (size_t)stage * plan.stage_floats;
    for (int ra = row0; ra < R; ra += 2 * RPC, ++pairs) {
      const int rb = ra + RPC;
      A xa[KP], xb[KP], ya[NQ], yb[NQ];
      {
        float va[KP * E], vb[KP * E], wa[NQ * E], wb[NQ * E];
        lds_n<KP * E>(tile + po + ra * pw, va);
        lds_n<KP * E>(tile + po + rb * pw, vb);
        if constexpr (E == 2) {  // 8-byte elements: 8-byte loads at any element offset
#pragma unroll
          for (int i = 0; i < NQ; ++i) {
            const float2 ta = *reinterpret_cast<const float2*>(tile + qo + ra * qs.bw + 2 * i);
            const float2 tb = *reinterpret_cast<const float2*>(tile + qo + rb * qs.bw + 2 * i);
            wa[2 * i] = ta.x;
            wa[2 * i + 1] = ta.y;
            wb[2 * i] = tb.x;
            wb[2 * i + 1] = tb.y;
          }
        } else if (qvec) {
          lds_n<NQ * E>(tile + qo + ra * qs.bw, wa);
          lds_n<NQ * E>(tile + qo + rb * qs.bw, wb);
        } else {
#pragma unroll
          for (int i = 0; i < NQ * E; ++i) {
            wa[i] = tile[qo + ra * qs.bw + i];
            wb[i] = tile[qo + rb * qs.bw + i];
          }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          xa[k] = elem<P>(va, k);
          xb[k] = elem<P>(vb, k);
        }
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
          ya[j] = elem<P>(wa, j);
          yb[j] = elem<P>(wb, j);
        }
      }
      if constexpr (kAnchored && kPack) {
        // running sums of squares: P columns in pairs where KP is even
        if constexpr (KP % 2 == 0) {
#pragma unroll
          for (int k = 0; k < KP; k += 2) {
            float2 v = x2::fma2(float2{xa[k], xa[k + 1]}, float2{xa[k], xa[k + 1]}, float2{sp[k], sp[k + 1]});
            v = x2::fma2(float2{xb[k], xb[k + 1]}, float2{xb[k], xb[k + 1]}, v);
            sp[k] = v.x;
            sp[k + 1] = v.y;
          }
        } else {
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            sp[k] = __fmaf_rn(xa[k], xa[k], sp[k]);
            sp[k] = __fmaf_rn(xb[k], xb[k], sp[k]);
          }
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          float2 v = x2::fma2(float2{ya[2 * h], ya[2 * h + 1]}, float2{ya[2 * h], ya[2 * h + 1]},
                              float2{sq[2 * h], sq[2 * h + 1]});
          v = x2::fma2(float2{yb[2 * h], yb[2 * h + 1]}, float2{yb[2 * h], yb[2 * h + 1]}, v);
          sq[2 * h] = v.x;
          sq[2 * h + 1] = v.y;
        }
        // anchors are raised rarely: one test of all thresholds keeps the
        // raises out of the common path
        bool raise = false;
#pragma unroll
        for (int k = 0; k < KP; ++k) raise |= sp[k] > ta[k];
#pragma unroll
        for (int j = 0; j < NQ; ++j) raise |= sq[j] > tb[j];
        if (raise) {
#pragma unroll
          for (int k = 0; k < KP; ++k)
            if (sp[k] > ta[k]) {
              const float a1 = anc_anchor(sp[k]);
#pragma unroll
              for (int h = 0; h < NH; ++h) {
                anc_move(s2[k][h].x, c2[k][h].x, an[k] * bn[2 * h], a1 * bn[2 * h]);
                anc_move(s2[k][h].y, c2[k][h].y, an[k] * bn[2 * h + 1], a1 * bn[2 * h + 1]);
              }
              an[k] = a1;
              ta[k] = a1 * a1 * (1.0f / 4.5f);
            }
#pragma unroll
          for (int j = 0; j < NQ; ++j)
            if (sq[j] > tb[j]) {
              const float b1 = anc_anchor(sq[j]);
#pragma unroll
              for (int k = 0; k < KP; ++k) {
                float& sv = (j & 1) ? s2[k][j >> 1].y : s2[k][j >> 1].x;
                float& cv = (j & 1) ? c2[k][j >> 1].y : c2[k][j >> 1].x;
                anc_move(sv, cv, an[k] * bn[j], an[k] * b1);
              }
              bn[j] = b1;
              tb[j] = b1 * b1 * (1.0f / 4.5f);
            }
        }
        // s' = fma(x, y, s), z = s' - s, e = fma(x, -y, z) = -d exactly,
        // c - e = c + d: the anchored update of the file header, two Q
        // columns per instruction
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float* xr = r == 0 ? xa : xb;
          const float* yr = r == 0 ? ya : yb;
          float2 y2[NH], yn[NH];
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            y2[h] = float2{yr[2 * h], yr[2 * h + 1]};
            yn[h] = x2::mul2(y2[h], neg1);
          }
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            const float2 xx{xr[k], xr[k]};
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              const float2 t = s2[k][h];
              s2[k][h] = x2::fma2(xx, y2[h], t);
              const float2 z = x2::sub2(s2[k][h], t);
              c2[k][h] = x2::sub2(c2[k][h], x2::fma2(xx, yn[h], z));
            }
          }
        }
        if ((pairs & 3) == 3) {  // every 8 rows: fold c into s (|s| >= |c|)
#pragma unroll
          for (int k = 0; k < KP; ++k)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              const float2 t = x2::add2(s2[k][h], c2[k][h]);
              c2[k][h] = x2::sub2(c2[k][h], x2::sub2(t, s2[k][h]));
              s2[k][h] = t;
            }
        }
      } else if constexpr (kAnchored) {
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          sp[k] = __fmaf_rn(hi_of(xa[k]), hi_of(xa[k]), sp[k]);
          sp[k] = __fmaf_rn(hi_of(xb[k]), hi_of(xb[k]), sp[k]);
        }
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
          sq[j] = __fmaf_rn(hi_of(ya[j]), hi_of(ya[j]), sq[j]);
          sq[j] = __fmaf_rn(hi_of(yb[j]), hi_of(yb[j]), sq[j]);
        }
        bool raise = false;  // as in the packed path: one test of all thresholds
#pragma unroll
        for (int k = 0; k < KP; ++k) raise |= sp[k] > ta[k];
#pragma unroll
        for (int j = 0; j < NQ; ++j) raise |= sq[j] > tb[j];
        if (raise) {
#pragma unroll
          for (int k = 0; k < KP; ++k)
            if (sp[k] > ta[k]) {
              const float a1 = anc_anchor(sp[k]);
#pragma unroll
              for (int j = 0; j < NQ; ++j) anc_move(sa[k][j], ca[k][j], an[k] * bn[j], a1 * bn[j]);
              an[k] = a1;
              ta[k] = a1 * a1 * (1.0f / 4.5f);
            }
#pragma unroll
          for (int j = 0; j < NQ; ++j)
            if (sq[j] > tb[j]) {
              const float b1 = anc_anchor(sq[j]);
#pragma unroll
              for (int k = 0; k < KP; ++k) anc_move(sa[k][j], ca[k][j], an[k] * bn[j], an[k] * b1);
              bn[j] = b1;
              tb[j] = b1 * b1 * (1.0f / 4.5f);
            }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
          for (int j = 0; j < NQ; ++j) {
            anc_add(sa[k][j], ca[k][j], xa[k], ya[j]);
            anc_add(sa[k][j], ca[k][j], xb[k], yb[j]);
          }
        if ((pairs & 3) == 3) {  // every 8 rows: fold c into s (|s| >= |c|)
#pragma unroll
          for (int k = 0; k < KP; ++k)
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
              const float t = __fadd_rn(sa[k][j], ca[k][j]);
              ca[k][j] = __fsub_rn(ca[k][j], __fsub_rn(t, sa[k][j]));
              sa[k][j] = t;
            }
        }
      } else if constexpr (kPack) {
        // Dot2 of two Q columns per instruction: the error terms come out
        // negated from the negated Q pair, built once per row
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const A* xr = r == 0 ? xa : xb;
          const A* yr = r == 0 ? ya : yb;
          float2 yh[NH], yl[NH], nyh[NH], nyl[NH];
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            yh[h] = float2{hi_of(yr[2 * h]), hi_of(yr[2 * h + 1])};
            yl[h] = float2{lo_of(yr[2 * h]), lo_of(yr[2 * h + 1])};
            nyh[h] = x2::mul2(yh[h], neg1);
            nyl[h] = x2::mul2(yl[h], neg1);
          }
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            const float2 xh{hi_of(xr[k]), hi_of(xr[k])}, xl{lo_of(xr[k]), lo_of(xr[k])};
#pragma unroll
            for (int h = 0; h < NH; ++h) x2::dot2x2(s2[k][h], c2[k][h], xh, xl, yh[h], nyh[h], nyl[h]);
          }
        }
        // renormalise every 2 rows (FastTwoSum)
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const float2 t = x2::add2(s2[k][h], c2[k][h]);
            c2[k][h] = x2::sub2(c2[k][h], x2::sub2(t, s2[k][h]));
            s2[k][h] = t;
          }
      } else {
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
          for (int j = 0; j < NQ; ++j) {
            dot2_add(sa[k][j], ca[k][j], xa[k], ya[j]);
            dot2_add(sa[k][j], ca[k][j], xb[k], yb[j]);
            const df t = fast_two_sum(sa[k][j], ca[k][j]);
            sa[k][j] = t.hi;
            ca[k][j] = t.lo;
          }
      }
    }
    // this warp is done with the stage; the last warp to finish refills it
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&arrived[stage], 1) == NW - 1) {
        arrived[stage] = 0;
        const long long nx = ch + (long long)NS * gridDim.x;
        if (nx < nchunks) {
          __threadfence_block();
          fence_proxy_async();
          issue(nx, stage);
        }
      }
    }
  }
  __syncthreads();
  const int pq = p * q;
  if (*fail) {
    // copies still in flight land in this CTA's shared memory: wait for them
    // (bounded) before leaving, then report NaN partial sums
    if (threadIdx.x == 0)
      for (int j = 0; j < NS; ++j) {
        const long long ch = blockIdx.x + (long long)(it + j) * gridDim.x;
        if (ch < nchunks) mbar_wait(&full[(it + j) % NS], (unsigned)(((it + j) / NS) & 1));
      }
    __syncthreads();
    for (int e = threadIdx.x; e < pq; e += kT) partial[(long long)blockIdx.x * pq + e] = df{__int_as_float(0x7fc00000), 0.f};
    return;
  }
  if constexpr (kPack) {
#pragma unroll
    for (int k = 0; k < KP; ++k)
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        sa[k][2 * h] = s2[k][h].x;
        sa[k][2 * h + 1] = s2[k][h].y;
        ca[k][2 * h] = c2[k][h].x;
        ca[k][2 * h + 1] = c2[k][h].y;
      }
  }
  df* red = reinterpret_cast<df*>(smem);
#pragma unroll
  for (int k = 0; k < KP; ++k)
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      df g;
      if constexpr (kAnchored) {
        g = two_sum(__fsub_rn(sa[k][j], an[k] * bn[j]), ca[k][j]);  // s - sigma is exact
      } else {
        g = fast_two_sum(sa[k][j], ca[k][j]);
      }
#pragma unroll
      for (int off = 16; off >= TPR; off >>= 1)
        g = df_add(g, df{__shfl_down_sync(0xffffffffu, g.hi, off), __shfl_down_sync(0xffffffffu, g.lo, off)});
      // the lane column's place in P and Q (prefix and padding columns are dropped)
      const TmaSeg& sg = plan.seg[sgl];
      const int e = pc0 + k - sg.pstart - sg.xe;
      const int c = sg.c0 + e;
      if (lane < TPR && e >= 0 && e < sg.nc && j < q) red[(warp * p + c) * q + j] = g;
    }
  __syncthreads();
  for (int e = threadIdx.x; e < pq; e += kT) {
    df v = red[e];
    for (int w = 1; w < NW; ++w) v = df_add(v, red[w * pq + e]);
    partial[(long long)blockIdx.x * pq + e] = v;
  }
}

// smallest w >= need, w a multiple of 4 floats, w = rho (mod 32) when rho > 0
int padded_width(int need, int rho) {
  int w = (need + 3) & ~3;
  if (rho > 0)
    while (w % 32 != rho) w += 4;
  return w;
}

template <class P, int TPR, int KP, int NQ>
cudaError_t run(const CUtensorMap (&maps)[kMaxSeg], const TmaPlan& plan, long long r0, long long r1, int p, int q,
                void* partial, int max_blocks, int* nblocks, cudaStream_t st) {
  auto kern = k_gram_tma<P, TPR, KP, NQ>;
  const size_t sm = (size_t)plan.bar_off * 4 + kBarBytes;
  // the opt-in is set once per kernel instance: to the largest plan allowed
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(kern), kMaxSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long nchunks = (r1 - r0 + plan.R - 1) / plan.R;
  long long g = std::min<long long>((long long)std::max(per_sm, 1) * std::max(sms, 1), max_blocks);
  g = std::max<long long>(1, std::min(g, nchunks));
  *nblocks = (int)g;
  kern<<<(int)g, kT, sm, st>>>(maps[0], maps[1], maps[2], maps[3], plan, r0, r1, p, q,
                               reinterpret_cast<df*>(partial));
  return cudaGetLastError();
}

template <class P, int TPR, int KP = 4>
cudaError_t run_q4(const CUtensorMap (&maps)[kMaxSeg], const TmaPlan& plan, long long r0, long long r1, int p, int q,
                   int nq, void* partial, int max_blocks, int* nb, cudaStream_t st) {
  if (nq <= 1) return run<P, TPR, KP, 1>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
  if (nq <= 2) return run<P, TPR, KP, 2>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
  return run<P, TPR, KP, 4>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
}

template <class P>
cudaError_t gram_tma_p(const SegV* segs, int nseg, SegV Q, long long r0, long long r1, int p, void* partial,
                       int max_blocks, int* nb, cudaStream_t st) {
  constexpr int E = P::id == kF32 ? 1 : 2;
  const int q = Q.nc;
  // elements between each block's 16-byte copy boundary and its first column
  int xe[kMaxSeg];
  for (int s = 0; s <= nseg; ++s) {
    const SegV& g = s < nseg ? segs[s] : Q;
    const uintptr_t a = reinterpret_cast<uintptr_t>(g.p);
    if (a % (4 * E) != 0 || (g.ld * (long long)(4 * E)) % 16 != 0) return cudaErrorNotSupported;
    xe[s] = (int)((a & uintptr_t(15)) / (4 * E));
  }
  // Q columns of the kernel instance and P columns per lane: a lane owns at
  // most 16 pairs, 4 P columns for up to 4 Q columns, else 2
  const int nq = q <= 1 ? 1 : q <= 2 ? 2 : q <= 4 ? 4 : 8;
  auto lane_cols = [&](int kp) {
    int pp = 0;
    for (int s = 0; s < nseg; ++s) pp += (xe[s] + segs[s].nc + kp - 1) / kp * kp;
    return pp;
  };
  int kp = nq <= 4 ? 4 : 2;
  int tpr = 2;
  while (tpr * kp < lane_cols(kp)) tpr *= 2;
  // 3 columns per lane where 16 lanes of 3 cover what 16 of 4 would leave a
  // quarter or more idle (32 < p <= 48)
  if (kp == 4 && tpr == 16 && lane_cols(3) <= 48 && lane_cols(4) <= 48) kp = 3;
  if (tpr > 32) return cudaErrorNotSupported;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // bank padding: the rows that one shared-memory wavefront reads start on
  // distinct banks (tpr kp E floats per row of lanes)
  const int rho = kp == 3 ? 0 : (tpr * kp * E) % 32;
  // tile rows of every block: lane columns, their first lane column and the
  // box width (the last P segment also covers the lane columns past it, Q its
  // xe prefix and nq columns)
  int ncpv[kMaxSeg], pstv[kMaxSeg], bwv[kMaxSeg];
  for (int s = 0, pstart = 0; s <= nseg; ++s) {
    const int nc = s < nseg ? segs[s].nc : q;
    ncpv[s] = s < nseg ? (xe[s] + nc + kp - 1) / kp * kp : nq;
    pstv[s] = pstart;
    const int cover = s == nseg - 1 ? tpr * kp - pstart : s < nseg ? ncpv[s] : xe[s] + nq;
    bwv[s] = padded_width(cover * E, s < nseg ? rho : std::max(4, nq * E) % 32);
    if (bwv[s] > 256) return cudaErrorNotSupported;
    if (s < nseg) pstart += ncpv[s];
  }
  // (rows per stage, stages): the first candidate whose ring lets two CTAs
  // share an SM, else the first that fits at all; more rows per stage spread
  // the stage hand-over over more rows, more stages keep more tiles in flight
  const int rpc = kT / tpr;
  const int cands[4][2] = {{std::min(8 * rpc, 256), 3}, {std::min(4 * rpc, 256), 4}, {2 * rpc, 4}, {2 * rpc, 3}};
  auto smem_of = [&](int R, int stages) {
    int soff = 0;
    for (int s = 0; s <= nseg; ++s) soff += (bwv[s] * R + 31) & ~31;
    const int red = (kT / 32) * p * q * (int)(sizeof(df) / 4);
    return (size_t)((std::max(stages * soff, red) + 31) & ~31) * 4 + kBarBytes;
  };
  int pick = -1;
  for (int pass = 0; pass < 2 && pick < 0; ++pass)
    for (int ci = 0; ci < 4 && pick < 0; ++ci)
      if (smem_of(cands[ci][0], cands[ci][1]) <= (size_t)(pass == 0 ? kRingTwoCtas : kMaxSmem)) pick = ci;
  if (pick < 0) return cudaErrorNotSupported;
  const int R = cands[pick][0];
  TmaPlan plan{};
  plan.nP = nseg;
  plan.R = R;
  plan.stages = cands[pick][1];
  CUtensorMap maps[kMaxSeg];
  std::memset(maps, 0, sizeof(maps));
  int soff = 0, c0 = 0;
  for (int s = 0; s <= nseg; ++s) {
    const SegV& g = s < nseg ? segs[s] : Q;
    const uintptr_t base = reinterpret_cast<uintptr_t>(g.p) & ~uintptr_t(15);
    const long long stride = g.ld * (long long)(4 * E);
    const int need = (xe[s] + g.nc) * E;  // floats of data from the copy boundary
    if (need * 4LL > stride) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)need, (cuuint64_t)r1};
    const cuuint64_t strides[1] = {(cuuint64_t)stride};
    const cuuint32_t box[2] = {(cuuint32_t)bwv[s], (cuuint32_t)R};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult cr = enc(&maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, reinterpret_cast<void*>(base), dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorNotSupported;
    plan.seg[s] = TmaSeg{soff, bwv[s], pstv[s], ncpv[s], xe[s], g.nc, c0};
    soff += (bwv[s] * R + 31) & ~31;
    if (s < nseg) c0 += g.nc;
  }
  plan.stage_floats = soff;
  {
    const int red = (kT / 32) * p * q * (int)(sizeof(df) / 4);
    plan.bar_off = (std::max(plan.stages * soff, red) + 31) & ~31;
  }
  if ((size_t)plan.bar_off * 4 + kBarBytes > (size_t)kMaxSmem) return cudaErrorNotSupported;
  for (int s = nseg + 1; s < kMaxSeg; ++s) maps[s] = maps[nseg];  // unused slots: any valid map
  if (kp == 3) return run_q4<P, 16, 3>(maps, plan, r0, r1, p, q, nq, partial, max_blocks, nb, st);
  if (kp == 4) {
    if (tpr == 2) return run_q4<P, 2>(maps, plan, r0, r1, p, q, nq, partial, max_blocks, nb, st);
    if (tpr == 4) return run_q4<P, 4>(maps, plan, r0, r1, p, q, nq, partial, max_blocks, nb, st);
    if (tpr == 8) return run_q4<P, 8>(maps, plan, r0, r1, p, q, nq, partial, max_blocks, nb, st);
    if (tpr == 16) return run_q4<P, 16>(maps, plan, r0, r1, p, q, nq, partial, max_blocks, nb, st);
    return run_q4<P, 32>(maps, plan, r0, r1, p, q, nq, partial, max_blocks, nb, st);
  }
  if (tpr == 2) return run<P, 2, 2, 8>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
  if (tpr == 4) return run<P, 4, 2, 8>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
  if (tpr == 8) return run<P, 8, 2, 8>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
  if (tpr == 16) return run<P, 16, 2, 8>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
  return run<P, 32, 2, 8>(maps, plan, r0, r1, p, q, partial, max_blocks, nb, st);
}

}  // namespace

cudaError_t launch_gram_tma(int prec, long long r0, long long r1, const SegV* P, int nseg, SegV Q, void* partial,
                            int max_blocks, int* nblocks, cudaStream_t st) {
  int p = 0;
  for (int s = 0; s < nseg; ++s) p += P[s].nc;
  if (nseg < 1 || nseg > 3 || p < 1 || p > kMaxP || Q.nc < 1 || Q.nc > 8 || r1 <= r0 || r1 > 2147483647LL)
    return cudaErrorNotSupported;
  if (prec == kF32) return gram_tma_p<PF32>(P, nseg, Q, r0, r1, p, partial, max_blocks, nblocks, st);
  if (prec == kDF64) return gram_tma_p<PDF64>(P, nseg, Q, r0, r1, p, partial, max_blocks, nblocks, st);
  return cudaErrorNotSupported;
}

}  // namespace phsvds
