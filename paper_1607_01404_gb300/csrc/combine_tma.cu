// TMA-fed basis update Out = alpha In + [P0 P1 P2] C, optionally followed by
// Out <- Out R^-1 (the Sec. 3.2 restart V <- V Z in place, the CGS update
// T <- T - V C and its CholQR scaling, the Ritz-vector combinations), for the
// F32 and DF64 storage modes, p <= 64 and q <= 32.
//
// Memory side, as in the TMA-fed Gram: row tiles of every P segment are
// streamed by cp.async.bulk.tensor.2d into a ring of shared-memory stages,
// one mbarrier per stage, and the last warp to finish a stage refills it with
// the CTA's next chunk.  A row of a tile belongs to one thread (F32) or to two
// threads in different warps, each with half of the outputs (double-float:
// half-height stages, so twice the stages fit in flight).  A thread reads its
// row from shared memory in 16-byte pieces (tile rows are padded to an odd
// number of 16-byte words, so the 8 rows of a quarter warp hit distinct
// banks), broadcasts the coefficients from shared memory and keeps its
// outputs in registers; its part of the In row (q columns or fewer) comes
// straight from global memory, loaded before the stage wait and added after
// the products, which keeps the ring for the wide P rows.  Columns past a
// segment's end arrive as zeros and meet zero coefficients, so the ragged row
// and column tails need no masks.
// Outputs go through a per-warp shared-memory buffer and leave as row
// segments: consecutive lanes store consecutive pieces of the warp's 32 rows
// (a few cache lines per store instruction instead of one line per lane, for
// rows whose stride is much wider than the q outputs); rows past L and
// columns past q are not written.
//
// In-place use (Out = P or Out = In, equal strides) is safe: a row is written
// only by the warp that owns it, after its tile has landed in shared memory,
// and later copies read other rows.
//
// Arithmetic: F32 multiply-adds in column order, then + In;
// DF64: Dot2 (Ogita, Rump and Oishi 2005) per output, the exact product of
// the high parts by FMA plus the cross terms, TwoSum into the high word and
// the rounding errors summed in the low word, In added by TwoSum and the sum
// renormalised once at the end (12 FP32 operations per product instead of 15
// for a renormalising double-float FMA).
//
// Every mbarrier wait is bounded; a CTA whose wait runs out writes NaN to all
// rows of its chunks, waits (bounded) for its copies in flight and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace phsvds {

namespace {

using namespace tma;

constexpr int kT = 256;          // threads per CTA
constexpr int kMaxStages = 6;
constexpr int kMaxSmem = 200 * 1024 + 128;
constexpr int kTwoCtas = 113 * 1024;  // a plan at most this large lets two CTAs share an SM
constexpr int kBarBytes = kMaxStages * 8 + kMaxStages * 4 + 16;

struct CmbSeg {
  int soff;    // float offset of the segment's tile inside a stage
  int bw;      // floats per tile row
  int ncp;     // columns read per row (nc rounded up to a 16-byte multiple)
  int pstart;  // coefficient row of column 0 in the padded coefficient table
  int nc;      // columns
  int c0;      // first column of the segment in P
};
struct CmbPlan {
  CmbSeg seg[3];
  int nP;
  int stage_floats;    // a multiple of 32
  int stages;
  int ppad;      // rows of the padded coefficient table
  int coef_off;  // float offsets of the coefficient table, R^-1, the warps'
  int rinv_off;  // output boxes and the barriers
  int obuf_off;
  int bar_off;
};

// Dot2 step: hi + lo += x c
__device__ __forceinline__ void dot2_step(float& hi, float& lo, df x, df c) {
  const df pr = two_prod(x.hi, c.hi);
  const float pl = __fmaf_rn(x.hi, c.lo, __fmaf_rn(x.lo, c.hi, pr.lo));
  const df s = two_sum(hi, pr.hi);
  hi = s.hi;
  lo = __fadd_rn(lo, __fadd_rn(s.lo, pl));
}

template <class P, int QT, int TPRW>
__global__ void __launch_bounds__(kT, ((QT / TPRW) * (P::id == kF32 ? 1 : 2) < 32) ? 2 : 1)
    k_combine_tma(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
                  const __grid_constant__ CUtensorMap m2, const CmbPlan plan, long long L, int q,
                  const typename P::C* __restrict__ coef, const typename P::C* __restrict__ Rinv,
                  const typename P::S* In, long long ldin, int in_vec, typename P::S* Out, long long ldout,
                  typename P::S* Out2, long long ldout2, int vw) {
  using C = typename P::C;
  constexpr bool kDF = P::id != kF32;
  constexpr int E = kDF ? 2 : 1;      // floats per element
  constexpr int W = 4 / E;            // elements per 16-byte piece
  constexpr int R = kT / TPRW;        // rows per stage
  constexpr int QH = QT / TPRW;       // outputs per thread
  constexpr int CV = QT * E / 4;      // 16-byte pieces of a coefficient row
  constexpr int CVH = QH * E / 4;     // ... of a thread's part of it
  constexpr int OBW = QH * E;         // floats of a thread's outputs
  constexpr int OBS = (OBW / 4) % 2 ? OBW : OBW + 4;  // their row stride in the output buffer (odd 16-byte words)
  constexpr int QR = QT <= 8 ? QT : 1;
  constexpr int NW = kT / 32;
  static_assert(QH * E % 4 == 0, "a thread's outputs must fill 16-byte pieces");
  extern __shared__ __align__(128) float smem[];
  float* cs = smem + plan.coef_off;
  float* rs = smem + plan.rinv_off;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + plan.bar_off);
  int* arrived = reinterpret_cast<int*>(full + kMaxStages);
  int* fail = arrived + kMaxStages;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int prow = threadIdx.x % R;  // row of the stage
  const int part = threadIdx.x / R;  // outputs part QH .. part QH + QH - 1 (warp-uniform)
  const int wrow0 = prow - lane;     // first stage row of this warp
  float* obuf = smem + plan.obuf_off + warp * 32 * OBS;
  const int NS = plan.stages;
  const long long nchunks = (L + R - 1) / R;
  // the segments' fields in registers (constant indices: a run-time index
  // into the parameter block would copy it to the stack)
  int s_soff[3], s_bw[3], s_ncp[3], s_pst[3], s_nc[3], s_c0[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s_soff[i] = plan.seg[i].soff;
    s_bw[i] = plan.seg[i].bw;
    s_ncp[i] = plan.seg[i].ncp;
    s_pst[i] = plan.seg[i].pstart;
    s_nc[i] = plan.seg[i].nc;
    s_c0[i] = plan.seg[i].c0;
  }
  unsigned tx_bytes = 0;
#pragma unroll
  for (int sg = 0; sg < 3; ++sg)
    if (sg < plan.nP) tx_bytes += (unsigned)(s_bw[sg] * R * 4);
  auto issue = [&](long long ch, int st) {
    float* base = smem + (size_t)st * plan.stage_floats;
    mbar_expect_tx(&full[st], tx_bytes);
    const int y = (int)(ch * R);
#pragma unroll
    for (int sg = 0; sg < 3; ++sg)
      if (sg < plan.nP) load_2d(base + s_soff[sg], sg == 0 ? &m0 : sg == 1 ? &m1 : &m2, 0, y, &full[st]);
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
  // the padded coefficient table: row pstart + c of segment sg holds P column
  // c0 + c (zeros for the padding columns and for outputs j >= q)
  {
    C* ct = reinterpret_cast<C*>(cs);
    for (int e = threadIdx.x; e < plan.ppad * QT; e += kT) {
      const int r = e / QT, j = e % QT;
      const int sg = (plan.nP > 1 && r >= s_pst[1]) ? ((plan.nP > 2 && r >= s_pst[2]) ? 2 : 1) : 0;
      const int pst = sg == 0 ? s_pst[0] : sg == 1 ? s_pst[1] : s_pst[2];
      const int nc = sg == 0 ? s_nc[0] : sg == 1 ? s_nc[1] : s_nc[2];
      const int cz = sg == 0 ? s_c0[0] : sg == 1 ? s_c0[1] : s_c0[2];
      const int c = r - pst;
      ct[e] = (c < nc && j < q) ? coef[(long long)(cz + c) * q + j] : C{};
    }
    if (QT <= 8 && Rinv) {
      C* rt = reinterpret_cast<C*>(rs);
      for (int e = threadIdx.x; e < QR * QR; e += kT) {
        const int i = e / QR, j = e % QR;
        rt[e] = (i < q && j < q) ? Rinv[i * q + j] : C{};
      }
    }
  }
  __syncthreads();

  const bool stores = part * QH < q;  // a part whose columns all lie past q stores nothing
  // In values of row prow of chunk ch for this thread's part (zeros past L or q)
  auto load_in = [&](long long ch, float (&dst)[OBW]) {
#pragma unroll
    for (int k = 0; k < OBW; ++k) dst[k] = 0.f;
    const long long r = ch * R + prow;
    const int nin = min(OBW, q * E - part * OBW);
    if (ch >= nchunks || r >= L || nin <= 0) return;
    const float* src = reinterpret_cast<const float*>(In) + r * ldin * E + part * OBW;
    if (in_vec && nin == OBW) {
#pragma unroll
      for (int v = 0; v < OBW / 4; ++v) {
        const float4 t = reinterpret_cast<const float4*>(src)[v];
        dst[4 * v] = t.x;
        dst[4 * v + 1] = t.y;
        dst[4 * v + 2] = t.z;
        dst[4 * v + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < OBW; ++k)
        if (k < nin) dst[k] = src[k];
    }
  };
  float inn[OBW];
#pragma unroll
  for (int k = 0; k < OBW; ++k) inn[k] = 0.f;
  if (In) load_in(blockIdx.x, inn);
  int it = 0;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++it) {
    const int stage = it % NS;
    // this thread's part of its In row, loaded from global memory one chunk
    // ahead (the load's latency overlaps a whole chunk) and added after the
    // products
    float inv[OBW];
#pragma unroll
    for (int k = 0; k < OBW; ++k) inv[k] = inn[k];
    if (In) load_in(ch + gridDim.x, inn);
    // warp-uniform decision: every lane of a warp leaves the loop together
    const bool ok = __all_sync(0xffffffffu, !*reinterpret_cast<volatile int*>(fail) && mbar_wait(&full[stage], (unsigned)((it / NS) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(fail, 1);
      break;
    }
    const float* tile = smem + (size_t)stage * plan.stage_floats;
    float hi[QH], lo[QH];
#pragma unroll
    for (int j = 0; j < QH; ++j) hi[j] = lo[j] = 0.f;
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
      if (sg >= plan.nP) break;
      const float4* row = reinterpret_cast<const float4*>(tile + s_soff[sg] + prow * s_bw[sg]);
      const float4* cb = reinterpret_cast<const float4*>(cs + s_pst[sg] * QT * E) + part * CVH;
      for (int c = 0; c < s_ncp[sg]; c += W) {
        const float4 xv = row[c / W];
        if constexpr (kDF) {
          const df x0{xv.x, xv.y}, x1{xv.z, xv.w};
#pragma unroll
          for (int v = 0; v < CVH; ++v) {
            const float4 c0 = cb[c * CV + v];
            dot2_step(hi[2 * v], lo[2 * v], x0, df{c0.x, c0.y});
            dot2_step(hi[2 * v + 1], lo[2 * v + 1], x0, df{c0.z, c0.w});
          }
#pragma unroll
          for (int v = 0; v < CVH; ++v) {
            const float4 c1 = cb[(c + 1) * CV + v];
            dot2_step(hi[2 * v], lo[2 * v], x1, df{c1.x, c1.y});
            dot2_step(hi[2 * v + 1], lo[2 * v + 1], x1, df{c1.z, c1.w});
          }
        } else {
          const float x[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
          for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int v = 0; v < CVH; ++v) {
              const float4 cv = cb[(c + w) * CV + v];
              hi[4 * v] = __fmaf_rn(x[w], cv.x, hi[4 * v]);
              hi[4 * v + 1] = __fmaf_rn(x[w], cv.y, hi[4 * v + 1]);
              hi[4 * v + 2] = __fmaf_rn(x[w], cv.z, hi[4 * v + 2]);
              hi[4 * v + 3] = __fmaf_rn(x[w], cv.w, hi[4 * v + 3]);
            }
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
    if constexpr (kDF) {
#pragma unroll
      for (int j = 0; j < QH; ++j) {
        const df a = two_sum(hi[j], inv[2 * j]);  // + In, then renormalise
        const df t = two_sum(a.hi, __fadd_rn(lo[j], __fadd_rn(a.lo, inv[2 * j + 1])));
        hi[j] = t.hi;
        lo[j] = t.lo;
      }
    } else {
#pragma unroll
      for (int j = 0; j < QH; ++j) hi[j] = __fadd_rn(hi[j], inv[j]);
    }
    if constexpr (QT <= 8 && TPRW == 1) {
      if (Rinv) {  // out_j = sum_{i <= j} out_i Rinv_ij, in place from the last column down
#pragma unroll
        for (int j = QT - 1; j >= 0; --j) {
          if constexpr (kDF) {
            const df* rt = reinterpret_cast<const df*>(rs);
            float th = 0.f, tl = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) dot2_step(th, tl, df{hi[i], lo[i]}, rt[i * QR + j]);
            const df t = two_sum(th, tl);
            hi[j] = t.hi;
            lo[j] = t.lo;
          } else {
            float t = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) t = __fmaf_rn(hi[i], rs[i * QR + j], t);
            hi[j] = t;
          }
        }
      }
    }
    // the warp's 32 rows x its part's columns go through the warp's output
    // buffer and leave as row segments, consecutive lanes on consecutive
    // pieces (a few cache lines per store instead of one line per lane)
    __syncwarp();  // the previous chunk's reads of the buffer are done
    float4* ob = reinterpret_cast<float4*>(obuf + lane * OBS);
#pragma unroll
    for (int v = 0; v < OBW / 4; ++v) {
      if constexpr (kDF)
        ob[v] = make_float4(hi[2 * v], lo[2 * v], hi[2 * v + 1], lo[2 * v + 1]);
      else
        ob[v] = make_float4(hi[4 * v], hi[4 * v + 1], hi[4 * v + 2], hi[4 * v + 3]);
    }
    __syncwarp();
    const long long y = ch * R + wrow0;
    if (stores && y < L) {
      const int nin = min(OBW, q * E - part * OBW);  // floats of this part inside the q columns
      const int npr = nin / vw;                      // pieces per row (vw divides nin)
      const int nrow = (int)min(32LL, L - y);
      for (int o = 0; o < 2; ++o) {
        float* dst = reinterpret_cast<float*>(o == 0 ? Out : Out2);
        if (!dst) break;
        const long long ld = (o == 0 ? ldout : ldout2) * E;
        dst += y * ld + part * OBW;
        for (int idx = lane; idx < nrow * npr; idx += 32) {
          const int rr = idx / npr, cc = (idx - rr * npr) * vw;
          const float* src = obuf + rr * OBS + cc;
          float* d = dst + rr * ld + cc;
          if (vw == 4)
            *reinterpret_cast<float4*>(d) = *reinterpret_cast<const float4*>(src);
          else if (vw == 2)
            *reinterpret_cast<float2*>(d) = *reinterpret_cast<const float2*>(src);
          else
            *d = *src;
        }
      }
    }
  }
  __syncthreads();
  if (*fail) {
    if (threadIdx.x == 0)
      for (int j = 0; j < NS; ++j) {
        const long long ch = blockIdx.x + (long long)(it + j) * gridDim.x;
        if (ch < nchunks) mbar_wait(&full[(it + j) % NS], (unsigned)(((it + j) / NS) & 1));
      }
    __syncthreads();
    const float nan = __int_as_float(0x7fc00000);
    if (part == 0)
      for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long long r = ch * R + prow;
        if (r >= L) continue;
        float* d = reinterpret_cast<float*>(Out + r * ldout);
        for (int e = 0; e < q * E; ++e) d[e] = nan;
      }
  }
}

// smallest width >= need floats, a multiple of 4, an odd number of 16-byte words
int odd_width(int need) {
  int w = (need + 3) & ~3;
  if ((w / 4) % 2 == 0) w += 4;
  return w;
}

// CTAs per SM of the plan: 0 = by the ring depth (PHSVDS_CMB_CTAS=1 or 2 forces one)
int forced_ctas() {
  static const int v = [] {
    const char* e = std::getenv("PHSVDS_CMB_CTAS");
    return e ? std::atoi(e) : 0;
  }();
  return v;
}

template <class P, int QT, int TPRW>
cudaError_t run(const CUtensorMap (&maps)[3], CmbPlan plan, long long L, int q, const void* coef, const void* Rinv,
                const void* In, long long ldin, int in_vec, void* Out, long long ldout, void* Out2, long long ldout2,
                int vw, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  constexpr int E = P::id == kF32 ? 1 : 2;
  constexpr int R = kT / TPRW;
  constexpr int OBW = QT / TPRW * E;
  constexpr int OBS = (OBW / 4) % 2 ? OBW : OBW + 4;
  auto kern = k_combine_tma<P, QT, TPRW>;
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(kern), kMaxSmem);
  if (e != cudaSuccess) return e;
  // the coefficient table, R^-1 and the output boxes follow the ring, the
  // barriers follow them
  auto layout = [&](int stages) {
    plan.stages = stages;
    plan.coef_off = stages * plan.stage_floats;
    plan.rinv_off = plan.coef_off + ((plan.ppad * QT * E + 31) & ~31);
    plan.obuf_off = plan.rinv_off + ((QT <= 8 && Rinv) ? ((QT * QT * E + 31) & ~31) : 0);
    plan.bar_off = plan.obuf_off + (kT / 32) * 32 * OBS;
    return (size_t)plan.bar_off * 4 + kBarBytes;
  };
  // two CTAs per SM when their rings keep at least 64 KB per SM in flight
  // (one stage per CTA is being consumed), else one CTA with the deepest ring
  const size_t stage_bytes = (size_t)plan.stage_floats * 4;
  const int force = forced_ctas();
  int stages = 0;
  if (force != 1)
    for (int s = kMaxStages; s >= 2 && !stages; --s)
      if (layout(s) <= (size_t)kTwoCtas && (force == 2 || 2 * (s - 1) * stage_bytes >= 64 * 1024)) stages = s;
  for (int s = kMaxStages; s >= 2 && !stages; --s)
    if (layout(s) <= (size_t)kMaxSmem) stages = s;
  if (!stages) return cudaErrorNotSupported;
  const size_t sm = layout(stages);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long nchunks = (L + R - 1) / R;
  const long long g = std::max<long long>(1, std::min<long long>((long long)std::max(per_sm, 1) * std::max(sms, 1),
                                                                 nchunks));
  kern<<<(int)g, kT, sm, st>>>(maps[0], maps[1], maps[2], plan, L, q, reinterpret_cast<const C*>(coef),
                               reinterpret_cast<const C*>(Rinv), reinterpret_cast<const S*>(In), ldin, in_vec,
                               reinterpret_cast<S*>(Out), ldout, reinterpret_cast<S*>(Out2), ldout2, vw);
  return cudaGetLastError();
}

template <class P, int TPRW>
cudaError_t combine_tma_t(long long L, const SegV* segs, int nseg, const void* coef, const void* In, long long ldin,
                          int alpha_one, void* Out, long long ldout, int q, const void* Rinv, void* Out2,
                          long long ldout2, cudaStream_t st) {
  constexpr int E = P::id == kF32 ? 1 : 2;
  constexpr int W = 4 / E;
  constexpr int SZ = 4 * E;
  constexpr int R = kT / TPRW;
  // outputs per thread (a bucket of q) and, from it, the output box width
  int qt = 32;
  for (int b : {4, 8, 12, 16, 20, 24, 32})
    if (q <= b && (b / TPRW) * E % 4 == 0) {
      qt = b;
      break;
    }
  const int obw = qt / TPRW * E;  // floats of a thread's outputs
  CmbPlan plan{};
  CUtensorMap maps[3];
  std::memset(maps, 0, sizeof(maps));
  plan.nP = nseg;
  int soff = 0, pstart = 0, c0 = 0;
  for (int s = 0; s < nseg; ++s) {
    const SegV& g = segs[s];
    if (reinterpret_cast<uintptr_t>(g.p) % 16 != 0 || (g.ld * SZ) % 16 != 0 || g.nc < 1 || g.ld < g.nc)
      return cudaErrorNotSupported;
    const int ncp = (g.nc + W - 1) / W * W;
    const int bw = odd_width(ncp * E);
    if (bw > 256) return cudaErrorNotSupported;
    if (!encode_rows(&maps[s], g.p, (long long)g.nc * E, L, g.ld * SZ, bw, R)) return cudaErrorNotSupported;
    plan.seg[s] = CmbSeg{soff, bw, ncp, pstart, g.nc, c0};
    soff += (bw * R + 31) & ~31;
    pstart += ncp;
    c0 += g.nc;
  }
  // In is read from global memory: 16-byte pieces when its rows allow them
  if (alpha_one && (!In || ldin < q || reinterpret_cast<uintptr_t>(In) % SZ != 0)) return cudaErrorNotSupported;
  const int in_vec = alpha_one && reinterpret_cast<uintptr_t>(In) % 16 == 0 && (ldin * SZ) % 16 == 0 ? 1 : 0;
  for (int s = nseg; s < 3; ++s) maps[s] = maps[0];
  // output pieces: the widest of 16, 8 or 4 bytes that divides every part's
  // floats inside the q columns, both strides and both base addresses
  int vw = 4;
  auto fits = [&](int w) {
    const int last = q * E - (q * E - 1) / obw * obw;  // floats of the last part with columns inside q
    const auto al = [&](const void* ptr, long long ld) {
      return reinterpret_cast<uintptr_t>(ptr) % (4 * w) == 0 && (ld * E) % w == 0;
    };
    return obw % w == 0 && last % w == 0 && al(Out, ldout) && (!Out2 || al(Out2, ldout2));
  };
  while (vw > 1 && !fits(vw)) vw /= 2;
  if (ldout < q || (Out2 && ldout2 < q)) return cudaErrorNotSupported;
  plan.stage_floats = soff;
  plan.ppad = pstart;
  // one thread per double-float row serves R^-1 only (q <= 8)
  constexpr int kMaxQT = (P::id == kDF64 && TPRW == 1) ? 8 : 32;
#define PHSVDS_CMB_TMA(QTV)                                                                              \
  if constexpr (QTV <= kMaxQT)                                                                            \
    if (qt == QTV)                                                                                        \
      return run<P, QTV, TPRW>(maps, plan, L, q, coef, Rinv, alpha_one ? In : nullptr, ldin, in_vec, Out, ldout, \
                               Out2, ldout2, vw, st);
  PHSVDS_CMB_TMA(4)
  PHSVDS_CMB_TMA(8)
  PHSVDS_CMB_TMA(12)
  PHSVDS_CMB_TMA(16)
  PHSVDS_CMB_TMA(20)
  PHSVDS_CMB_TMA(24)
  PHSVDS_CMB_TMA(32)
#undef PHSVDS_CMB_TMA
  return cudaErrorNotSupported;
}

// ---------------------------------------------------------------------------
// TMA-fed Ritz vectors and residuals (Sec. 3.3 residual kernel):
// X = V Y, R = W Y - X diag(theta), T = diag(dscale) R (optional), and per-CTA
// FP64-class partial sums of ||R_j||^2.  V and W row tiles share one ring
// stage; a row belongs to NP threads (one per group of QH output columns: one
// thread per row for F32, one per column for double-float, whose Dot2 work
// per row is 12 times larger and wants more warps in flight).
// ---------------------------------------------------------------------------
constexpr int kTR = 128;  // threads per CTA of the Ritz kernel

struct RitzPlan {
  int bw;            // floats per tile row of V and of W
  int ncp;           // columns read per row (g rounded up to a 16-byte multiple)
  int stage_floats;  // V tile then W tile, each a multiple of 32 floats
  int stages;
  int coef_off, red_off, bar_off;  // float offsets of Y and theta, the norm reduction, the barriers
};

template <class P, int QH, int NP>
__global__ void __launch_bounds__(kTR)
    k_ritz_tma(const __grid_constant__ CUtensorMap mv, const __grid_constant__ CUtensorMap mw, const RitzPlan plan,
               long long L, int g, int nb, const typename P::C* __restrict__ Y, const typename P::C* __restrict__ theta,
               typename P::S* X, typename P::S* Rr, long long ldb, const typename P::S* __restrict__ dscale,
               typename P::S* T, int vst, df* __restrict__ partial) {
  using C = typename P::C;
  using A = typename P::A;
  constexpr bool kDF = P::id != kF32;
  constexpr int E = kDF ? 2 : 1;
  constexpr int W = 4 / E;           // elements per 16-byte piece
  constexpr int R = kTR / NP;        // rows per stage
  constexpr int NBT = QH * NP;       // output columns of the table (nb padded)
  constexpr int NW = kTR / 32;
  static_assert(R % 32 == 0, "a warp's threads share one output part");
  extern __shared__ __align__(128) float smem[];
  C* ys = reinterpret_cast<C*>(smem + plan.coef_off);  // g padded rows x NBT, then theta (NBT)
  C* th = ys + plan.ncp * NBT;
  df* red = reinterpret_cast<df*>(smem + plan.red_off);  // NW x QH
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + plan.bar_off);
  int* arrived = reinterpret_cast<int*>(full + kMaxStages);
  int* fail = arrived + kMaxStages;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int prow = threadIdx.x % R;
  const int part = threadIdx.x / R;  // output columns part QH .. part QH + QH - 1 (warp-uniform)
  const int j0 = part * QH;
  const int NS = plan.stages;
  const long long nchunks = (L + R - 1) / R;
  const unsigned tx_bytes = (unsigned)(2 * plan.bw * R * 4);
  auto issue = [&](long long ch, int st) {
    float* base = smem + (size_t)st * plan.stage_floats;
    mbar_expect_tx(&full[st], tx_bytes);
    const int y = (int)(ch * R);
    load_2d(base, &mv, 0, y, &full[st]);
    load_2d(base + plan.stage_floats / 2, &mw, 0, y, &full[st]);
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
  for (int e = threadIdx.x; e < plan.ncp * NBT; e += kTR) {
    const int c = e / NBT, j = e % NBT;
    ys[e] = (c < g && j < nb) ? Y[(long long)c * nb + j] : C{};
  }
  for (int j = threadIdx.x; j < NBT; j += kTR) th[j] = j < nb ? theta[j] : C{};
  __syncthreads();
  A thv[QH];
#pragma unroll
  for (int jj = 0; jj < QH; ++jj) thv[jj] = th[j0 + jj];
  df nrm[QH];
#pragma unroll
  for (int jj = 0; jj < QH; ++jj) nrm[jj] = df{0.f, 0.f};

  int it = 0;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++it) {
    const int stage = it % NS;
    const bool ok = __all_sync(0xffffffffu, !*reinterpret_cast<volatile int*>(fail) &&
                                                mbar_wait(&full[stage], (unsigned)((it / NS) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(fail, 1);
      break;
    }
    const long long r = ch * R + prow;
    A dr{};
    if (T && r < L) dr = P::load(dscale + r);
    const float* tile = smem + (size_t)stage * plan.stage_floats;
    const float4* vrow = reinterpret_cast<const float4*>(tile + prow * plan.bw);
    const float4* wrow = reinterpret_cast<const float4*>(tile + plan.stage_floats / 2 + prow * plan.bw);
    float xh[QH], xl[QH], zh[QH], zl[QH];  // X = V Y and Z = W Y (low words: double-float only)
#pragma unroll
    for (int jj = 0; jj < QH; ++jj) xh[jj] = xl[jj] = zh[jj] = zl[jj] = 0.f;
    for (int c = 0; c < plan.ncp; c += W) {
      const float4 a = vrow[c / W], b = wrow[c / W];
      if constexpr (kDF) {
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          const df xv = w == 0 ? df{a.x, a.y} : df{a.z, a.w};
          const df wv = w == 0 ? df{b.x, b.y} : df{b.z, b.w};
          const C* yr = ys + (c + w) * NBT + j0;
#pragma unroll
          for (int jj = 0; jj < QH; ++jj) {
            const df y = yr[jj];
            dot2_step(xh[jj], xl[jj], xv, y);
            dot2_step(zh[jj], zl[jj], wv, y);
          }
        }
      } else {
        const float xv[4] = {a.x, a.y, a.z, a.w}, wv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float* yr = reinterpret_cast<const float*>(ys) + (c + w) * NBT + j0;
          float y[QH];
          if constexpr (QH % 4 == 0) {
#pragma unroll
            for (int v = 0; v < QH / 4; ++v) {
              const float4 t = reinterpret_cast<const float4*>(yr)[v];
              y[4 * v] = t.x;
              y[4 * v + 1] = t.y;
              y[4 * v + 2] = t.z;
              y[4 * v + 3] = t.w;
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < QH; ++jj) y[jj] = yr[jj];
          }
#pragma unroll
          for (int jj = 0; jj < QH; ++jj) {
            xh[jj] = __fmaf_rn(xv[w], y[jj], xh[jj]);
            zh[jj] = __fmaf_rn(wv[w], y[jj], zh[jj]);
          }
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
    if (r < L) {
      A xo[QH], ro[QH];
#pragma unroll
      for (int jj = 0; jj < QH; ++jj) {
        if constexpr (kDF) {
          const df xd = two_sum(xh[jj], xl[jj]);
          const df zd = two_sum(zh[jj], zl[jj]);
          xo[jj] = xd;
          ro[jj] = df_add(zd, df_neg(df_mul(xd, thv[jj])));
        } else {
          xo[jj] = xh[jj];
          ro[jj] = P::sub(zh[jj], P::mulc(xh[jj], thv[jj]));
        }
        if (j0 + jj < nb) nrm[jj] = P::gfma(nrm[jj], ro[jj], ro[jj]);
      }
      // stores: 16-byte pieces of this thread's columns where they all lie
      // inside nb and the rows allow them, else element by element
      typename P::S* xd = X + r * ldb + j0;
      typename P::S* rd = Rr + r * ldb + j0;
      typename P::S* td = T ? T + r * ldb + j0 : nullptr;
      if (vst && j0 + QH <= nb && (QH * E) % 4 == 0) {
#pragma unroll
        for (int v = 0; v < QH * E / 4; ++v) {
          float4 fx, fr, ft;
          if constexpr (kDF) {
            fx = make_float4(xo[2 * v].hi, xo[2 * v].lo, xo[2 * v + 1].hi, xo[2 * v + 1].lo);
            fr = make_float4(ro[2 * v].hi, ro[2 * v].lo, ro[2 * v + 1].hi, ro[2 * v + 1].lo);
          } else {
            fx = make_float4(xo[4 * v], xo[4 * v + 1], xo[4 * v + 2], xo[4 * v + 3]);
            fr = make_float4(ro[4 * v], ro[4 * v + 1], ro[4 * v + 2], ro[4 * v + 3]);
          }
          reinterpret_cast<float4*>(xd)[v] = fx;
          reinterpret_cast<float4*>(rd)[v] = fr;
          if (td) {
            if constexpr (kDF) {
              const df t0 = df_mul(dr, ro[2 * v]), t1 = df_mul(dr, ro[2 * v + 1]);
              ft = make_float4(t0.hi, t0.lo, t1.hi, t1.lo);
            } else {
              ft = make_float4(dr * ro[4 * v], dr * ro[4 * v + 1], dr * ro[4 * v + 2], dr * ro[4 * v + 3]);
            }
            reinterpret_cast<float4*>(td)[v] = ft;
          }
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < QH; ++jj)
          if (j0 + jj < nb) {
            P::store(xd + jj, xo[jj]);
            P::store(rd + jj, ro[jj]);
            if (td) {
              if constexpr (kDF)
                P::store(td + jj, df_mul(dr, ro[jj]));
              else
                P::store(td + jj, dr * ro[jj]);
            }
          }
      }
    }
  }
  __syncthreads();
  if (*fail) {
    if (threadIdx.x == 0)
      for (int j = 0; j < NS; ++j) {
        const long long ch = blockIdx.x + (long long)(it + j) * gridDim.x;
        if (ch < nchunks) mbar_wait(&full[(it + j) % NS], (unsigned)(((it + j) / NS) & 1));
      }
    if ((int)threadIdx.x < nb) partial[(long long)blockIdx.x * nb + threadIdx.x] = df{__int_as_float(0x7fc00000), 0.f};
    return;
  }
  // norms: the warp's rows, then the warps of each part in order
#pragma unroll
  for (int jj = 0; jj < QH; ++jj) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
      nrm[jj] = df_add(nrm[jj], df{__shfl_down_sync(0xffffffffu, nrm[jj].hi, o),
                                   __shfl_down_sync(0xffffffffu, nrm[jj].lo, o)});
    if (lane == 0) red[warp * QH + jj] = nrm[jj];
  }
  __syncthreads();
  if ((int)threadIdx.x < nb) {
    const int j = threadIdx.x, pj = j / QH, jj = j % QH;
    constexpr int WPP = R / 32;  // warps per part
    df v = red[(pj * WPP) * QH + jj];
    for (int w = 1; w < WPP; ++w) v = df_add(v, red[(pj * WPP + w) * QH + jj]);
    partial[(long long)blockIdx.x * nb + j] = v;
  }
}

template <class P, int QH, int NP>
cudaError_t ritz_run(long long L, const SegV& V, const SegV& Wm, int g, const void* Y, const void* theta, void* X,
                     void* Rr, long long ldb, int nb, const void* dscale, void* T, void* partial, int max_blocks,
                     int* nblocks, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  constexpr int E = P::id == kF32 ? 1 : 2;
  constexpr int W = 4 / E;
  constexpr int SZ = 4 * E;
  constexpr int R = kTR / NP;
  constexpr int NBT = QH * NP;
  for (const SegV* s : {&V, &Wm})
    if (reinterpret_cast<uintptr_t>(s->p) % 16 != 0 || (s->ld * SZ) % 16 != 0 || s->ld < g)
      return cudaErrorNotSupported;
  RitzPlan plan{};
  plan.ncp = (g + W - 1) / W * W;
  plan.bw = odd_width(plan.ncp * E);
  if (plan.bw > 256) return cudaErrorNotSupported;
  CUtensorMap mv, mw;
  if (!encode_rows(&mv, V.p, (long long)g * E, L, V.ld * SZ, plan.bw, R) ||
      !encode_rows(&mw, Wm.p, (long long)g * E, L, Wm.ld * SZ, plan.bw, R))
    return cudaErrorNotSupported;
  plan.stage_floats = 2 * ((plan.bw * R + 31) & ~31);
  auto layout = [&](int stages) {
    plan.stages = stages;
    plan.coef_off = stages * plan.stage_floats;
    plan.red_off = plan.coef_off + (((plan.ncp * NBT + NBT) * (int)sizeof(C) / 4 + 31) & ~31);
    plan.bar_off = plan.red_off + (((kTR / 32) * QH * (int)sizeof(df) / 4 + 31) & ~31);
    return (size_t)plan.bar_off * 4 + kBarBytes;
  };
  // the most CTAs per SM (up to 4) whose rings hold at least 3 stages, else
  // one CTA with the deepest ring
  int stages = 0;
  for (int c = 4; c >= 1 && !stages; --c)
    for (int s = kMaxStages; s >= 3 && !stages; --s)
      if (layout(s) <= (size_t)kMaxSmem && layout(s) * c + 1024 * c <= 228 * 1024) stages = s;
  if (!stages)
    for (int s = kMaxStages; s >= 2 && !stages; --s)
      if (layout(s) <= (size_t)kMaxSmem) stages = s;
  if (!stages) return cudaErrorNotSupported;
  const size_t sm = layout(stages);
  auto kern = k_ritz_tma<P, QH, NP>;
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(kern), kMaxSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTR, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long nchunks = (L + R - 1) / R;
  long long grid = std::min<long long>((long long)std::max(per_sm, 1) * std::max(sms, 1), nchunks);
  grid = std::max<long long>(1, std::min<long long>(grid, max_blocks));
  *nblocks = (int)grid;
  const auto al = [&](const void* ptr) { return !ptr || reinterpret_cast<uintptr_t>(ptr) % 16 == 0; };
  const int vst = al(X) && al(Rr) && al(T) && (ldb * SZ) % 16 == 0 ? 1 : 0;
  kern<<<(int)grid, kTR, sm, st>>>(mv, mw, plan, L, g, nb, reinterpret_cast<const C*>(Y),
                                   reinterpret_cast<const C*>(theta), reinterpret_cast<S*>(X), reinterpret_cast<S*>(Rr),
                                   ldb, reinterpret_cast<const S*>(dscale), reinterpret_cast<S*>(T), vst,
                                   reinterpret_cast<df*>(partial));
  return cudaGetLastError();
}

bool tma_combine_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("PHSVDS_COMBINE_TMA");
    return !(v && v[0] == '0');
  }();
  return on;
}

}  // namespace

cudaError_t launch_ritz_tma(int prec, long long L, SegV V, SegV W, int g, const void* Y, const void* theta, void* X,
                            void* R, long long ldb, int nb, const void* dscale, void* T, void* partial,
                            int max_blocks, int* nblocks, cudaStream_t st) {
  if (!tma_combine_enabled()) return cudaErrorNotSupported;
  if (g < 1 || g > 64 || nb < 1 || nb > 8 || L < 1 || L > (long long)INT_MAX - kTR || max_blocks < 1)
    return cudaErrorNotSupported;
  // F32: one thread per row with all nb outputs; double-float: one thread per
  // output column
  if (prec == kF32) {
    if (nb <= 4) return ritz_run<PF32, 4, 1>(L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, partial, max_blocks,
                                             nblocks, st);
    return ritz_run<PF32, 8, 1>(L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, partial, max_blocks, nblocks, st);
  }
  if (prec == kDF64) {
    if (nb <= 4) return ritz_run<PDF64, 1, 4>(L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, partial, max_blocks,
                                              nblocks, st);
    return ritz_run<PDF64, 2, 4>(L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, partial, max_blocks, nblocks, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_combine_tma(int prec, long long L, const SegV* P, int nseg, const void* coef, const void* In,
                               long long ldin, int alpha_one, void* Out, long long ldout, int q, const void* Rinv,
                               void* Out2, long long ldout2, cudaStream_t st) {
  if (!tma_combine_enabled()) return cudaErrorNotSupported;
  int p = 0;
  for (int s = 0; s < nseg; ++s) p += P[s].nc;
  if (nseg < 1 || nseg > 3 || p < 1 || p > 64 || q < 1 || q > 32 || (Rinv && q > 8) || L < 1 ||
      L > (long long)INT_MAX - kT)
    return cudaErrorNotSupported;
  // F32: one thread per row; double-float: two threads per row (half the
  // outputs each, half-height stages: twice the stages in flight for the same
  // shared memory) unless R^-1 needs all of a row's outputs in one thread
  if (prec == kF32)
    return combine_tma_t<PF32, 1>(L, P, nseg, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
  if (prec == kDF64) {
    if (Rinv)
      return combine_tma_t<PDF64, 1>(L, P, nseg, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
    return combine_tma_t<PDF64, 2>(L, P, nseg, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace phsvds
