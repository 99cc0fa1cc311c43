// pair_body.cuh -- sphere placement and the self-collision map-reduce
// (Sec. 6.2), one warp per configuration (device code shared by the
// single-robot and the batched pair kernels).
//
// A warp stages its configuration's world link poses (config-major, written by
// the tree kernel) into shared memory with vector loads, places the spheres
// (c_s = R_l c_local + p_l, Sec. 6.1.1) as SoA arrays -- column copies x, y,
// z, N = |c|^2 - r^2 and row copies pre-scaled by -2 -- and writes the
// sphere output.  The pair blocks (4x4 sphere groups, dealt by the host so
// that the 8 lanes of a shared-memory phase read distinct bank groups, rows
// kept per lane in runs) are then screened with
//   e = |c_i - c_j|^2 - t^2,  t = T_i + r_j,  T_i = max(best + r_i + margin, -r_min),
// expanded as (|c_i|^2 - T_i^2) + (|c_j|^2 - r_j^2) - 2 c_i . c_j - 2 T_i r_j
// (one add and four fused multiply-adds per pair); e < 0 exactly when
// |c_i - c_j| < t.  Raising T_i to -r_min only widens the screen, and keeps
// t >= 0 so that t^2 is monotone.
// best is the warp-wide running minimum, refreshed every two rounds with one
// integer min-reduction over an order-preserving key, so the exact path --
// sqrt distance, pair index, lexicographic (d, index) compare -- only runs
// for screened-in pairs, one candidate at a time.  The screen fires on
// e < etol, a host bound on the float rounding of the expanded form, so it
// never drops a pair the exact path would keep.  A 5-step shuffle reduction
// of (d, index) finishes the configuration: one configuration never spans
// more than one warp, so the paper's second reduce kernel becomes a register
// reduction.
#pragma once

#include "spatial.cuh"

#include <cuda_fp16.h>

#include <climits>

namespace wbe {

__host__ __device__ constexpr int a32(int x) { return (x + 31) & ~31; }

struct PairPlan {  // per warp, 32-bit words
  int xr, yr, zr, xc, yc, zc, nn, gb, q, bits, total;
  __host__ __device__ int ra_words() const { return xc; }  // the row (and pose) region
  __host__ __device__ PairPlan(int n, int Sg, int P, bool with_bits) {
    const int m = a32(4 * Sg);
    const int ra = 3 * m > a32(12 * n) ? 3 * m : a32(12 * n);  // rows; poses while staging
    xr = 0;
    yr = m;
    zr = 2 * m;
    xc = ra;
    yc = ra + m;
    zc = ra + 2 * m;
    nn = ra + 3 * m;
    gb = ra + 4 * m;  // group bounding spheres (float4 per group), culling only
    q = gb + m;       // queue of surviving schedule entries (64), culling only
    bits = q + 64;
    total = bits + (with_bits ? a32((P + 31) / 32) : 0);
  }
};

inline size_t pair_smem(const DevRobot& r, int warps, bool bits) {
  return sizeof(float) *
         ((size_t)a32(4 * r.Sg) + (size_t)warps * PairPlan(r.n, r.Sg, r.P, bits).total);
}

// order-preserving map of a float to a signed int (and back)
__device__ __forceinline__ int fkey(float f) {
  const int i = __float_as_int(f);
  return i < 0 ? i ^ 0x7FFFFFFF : i;
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k < 0 ? k ^ 0x7FFFFFFF : k); }

__device__ __forceinline__ float4 lds4(const char* base, uint32_t off) {
  return *reinterpret_cast<const float4*>(base + off);
}
__device__ __forceinline__ float pick(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// c_i - c_j of pair p from the placed sphere centres (zero when there is no
// pair): the vector the backward sweep needs for the worst pair's gradient
__device__ __forceinline__ void pair_diff(const DevRobot& r, const FwdArgs& A, int64_t b, int p,
                                          const float* xc, const float* yc, const float* zc) {
  float d[3] = {0.0f, 0.0f, 0.0f};
  if (p >= 0) {
    const int2 ij = __ldg(r.pairs + p);
    d[0] = xc[ij.x] - xc[ij.y];
    d[1] = yc[ij.x] - yc[ij.y];
    d[2] = zc[ij.x] - zc[ij.y];
  }
  A.wdiff[3 * b] = d[0];
  A.wdiff[3 * b + 1] = d[1];
  A.wdiff[3 * b + 2] = d[2];
}

template <bool FULL, bool BITS>
__device__ __forceinline__ void pair_one(const DevRobot& r, const PairSchedule32& ps,
                                         const FwdArgs& A, int64_t b, float* ws,
                                         const float4* radw, int lane) {
  const PairPlan pl(r.n, r.Sg, r.P, BITS);
  float* xr = ws + pl.xr;
  float* yr = ws + pl.yr;
  float* zr = ws + pl.zr;
  float* xc = ws + pl.xc;
  float* yc = ws + pl.yc;
  float* zc = ws + pl.zc;
  float* nn = ws + pl.nn;
  uint32_t* bm = reinterpret_cast<uint32_t*>(ws + pl.bits);
  const char* cxr = reinterpret_cast<const char*>(xr);
  const char* cyr = reinterpret_cast<const char*>(yr);
  const char* czr = reinterpret_cast<const char*>(zr);
  const char* cxc = reinterpret_cast<const char*>(xc);
  const char* cyc = reinterpret_cast<const char*>(yc);
  const char* czc = reinterpret_cast<const char*>(zc);
  const char* cnn = reinterpret_cast<const char*>(nn);
  const char* crad = reinterpret_cast<const char*>(radw);
  const int n = r.n, S = r.S;
  const int W = (r.P + 31) >> 5;
  const float margin = r.margin, etol = r.etol, nrmin = -r.rmin;
  const int rounds = ps.rounds;
  // ---- stage the link poses (contiguous), then place the spheres ----
  {
    const float4* src = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
    float4* dst = reinterpret_cast<float4*>(xr);
#pragma unroll 4
    for (int i = lane; i < 3 * n; i += 32) dst[i] = __ldg(src + i);
  }
  __syncwarp();
  for (int s = lane; s < 4 * r.Sg; s += 32) {
    float c[3] = {0.0f, 0.0f, 0.0f};
    float rs = 0.0f;
    if (s < S) {
      const float4 sp = __ldg(r.sph + s);
      // the link's staged pose as three vector loads (48-byte rows)
      const float4* P4 = reinterpret_cast<const float4*>(xr) + 3 * __ldg(r.sph_link + s);
      const float4 p0 = P4[0], p1 = P4[1], p2 = P4[2];
      const float P[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
      const float cl[3] = {sp.x, sp.y, sp.z};
      rot(P, cl, c);
      c[0] += P[9];
      c[1] += P[10];
      c[2] += P[11];
      rs = sp.w;
      if (A.sph) {
        float* o = A.sph + (b * S + s) * 3;
        o[0] = c[0];
        o[1] = c[1];
        o[2] = c[2];
      }
    }
    xc[s] = c[0];
    yc[s] = c[1];
    zc[s] = c[2];
    nn[s] = fmaf(-rs, rs, fmaf(c[2], c[2], fmaf(c[1], c[1], c[0] * c[0])));  // |c|^2 - r^2
  }
  __syncwarp();
  for (int s = lane; s < 4 * r.Sg; s += 32) {  // row copies, pre-scaled by -2
    xr[s] = -2.0f * xc[s];
    yr[s] = -2.0f * yc[s];
    zr[s] = -2.0f * zc[s];
  }
  if (BITS)
    for (int w = lane; w < W; w += 32) bm[w] = 0u;
  __syncwarp();
  if (!A.dmin && !BITS) return;  // sphere placement only
  if (rounds == 0) {
    if (lane == 0 && A.dmin) {
      A.dmin[b] = __int_as_float(0x7f800000);
      A.worst[b] = -1;
      if (A.wdiff) pair_diff(r, A, b, -1, xc, yc, zc);
    }
    if (BITS)
      for (int w = lane; w < W; w += 32) A.bits[b * (int64_t)W + w] = 0u;
    return;
  }
  float best = 1e15f;
  int bidx = INT_MAX;
  uint2 nxt = __ldg(ps.ent + lane);
  // seed: the exact distance of one pair of the lane's first block
  if (FULL && (nxt.y >> 16) != 0u) {
    const uint32_t ro = nxt.x & 0xFFFF, co = nxt.x >> 16;
    const float* pi = reinterpret_cast<const float*>(cxc + ro);
    const float* pj = reinterpret_cast<const float*>(cxc + co);
    const float d2 = dist2(pi[0], *reinterpret_cast<const float*>(cyc + ro),
                           *reinterpret_cast<const float*>(czc + ro), pj[0],
                           *reinterpret_cast<const float*>(cyc + co),
                           *reinterpret_cast<const float*>(czc + co));
    best = sqrtf(d2) - (lds4(crad, ro).x + lds4(crad, co).x);
    bidx = 16 * (nxt.y & 0xFFFF);
  }
  float gbest = fkey_inv(__reduce_min_sync(0xffffffffu, fkey(best)));
  uint32_t cur = 0xFFFFFFFFu;
  float4 XR = {}, YR = {}, ZR = {}, RR = {}, CC = {};
  float Ai[4], ti2[4];
  auto set_row = [&]() {
    const float bb = fminf(best, gbest) + margin;
    const float T0 = fmaxf(bb + RR.x, nrmin), T1 = fmaxf(bb + RR.y, nrmin);
    const float T2 = fmaxf(bb + RR.z, nrmin), T3 = fmaxf(bb + RR.w, nrmin);
    Ai[0] = fmaf(-T0, T0, CC.x);
    Ai[1] = fmaf(-T1, T1, CC.y);
    Ai[2] = fmaf(-T2, T2, CC.z);
    Ai[3] = fmaf(-T3, T3, CC.w);
    ti2[0] = -2.0f * T0;
    ti2[1] = -2.0f * T1;
    ti2[2] = -2.0f * T2;
    ti2[3] = -2.0f * T3;
  };
  for (int rr = 0; rr < rounds; ++rr) {
    const uint2 e = nxt;
    nxt = __ldg(ps.ent + (rr + 1) * 32 + lane);  // the schedule has a null round at the end
    const uint32_t ro = e.x & 0xFFFF, co = e.x >> 16;
    const uint32_t mask = e.y >> 16;
    if (ro != cur) {
      cur = ro;
      XR = lds4(cxr, ro);
      YR = lds4(cyr, ro);
      ZR = lds4(czr, ro);
      RR = lds4(crad, ro);
      const float4 N = lds4(cnn, ro);
      CC = make_float4(fmaf(RR.x, RR.x, N.x), fmaf(RR.y, RR.y, N.y), fmaf(RR.z, RR.z, N.z),
                       fmaf(RR.w, RR.w, N.w));  // |c_i|^2
      set_row();
    }
    const float4 X = lds4(cxc, co), Y = lds4(cyc, co), Z = lds4(czc, co), N = lds4(cnn, co),
                 Rc = lds4(crad, co);
    const float xr4[4] = {XR.x, XR.y, XR.z, XR.w}, yr4[4] = {YR.x, YR.y, YR.z, YR.w},
                zr4[4] = {ZR.x, ZR.y, ZR.z, ZR.w};
    const float xj[4] = {X.x, X.y, X.z, X.w}, yj[4] = {Y.x, Y.y, Y.z, Y.w},
                zj[4] = {Z.x, Z.y, Z.z, Z.w}, nj[4] = {N.x, N.y, N.z, N.w},
                rj[4] = {Rc.x, Rc.y, Rc.z, Rc.w};
    // e(a, c) = |c_a - c_c|^2 - t^2 with t = T_a + r_c, expanded
    auto screen = [&](int a, int c) {
      return fmaf(ti2[a], rj[c],
                  fmaf(zr4[a], zj[c], fmaf(yr4[a], yj[c], fmaf(xr4[a], xj[c], Ai[a] + nj[c]))));
    };
    float m;
    if (FULL) {
      float m4[4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
        m4[a] = fminf(fminf(screen(a, 0), screen(a, 1)), fminf(screen(a, 2), screen(a, 3)));
      m = fminf(fminf(m4[0], m4[1]), fminf(m4[2], m4[3]));
      m = mask ? m : __int_as_float(0x7f800000);  // null entries at the schedule's tail
    } else {
      m = __int_as_float(0x7f800000);
#pragma unroll
      for (int t = 0; t < 16; ++t)
        if ((mask >> t) & 1u) m = fminf(m, screen(t >> 2, t & 3));
    }
    if (m < etol) {
      // candidates of this block, then the exact path one at a time
      uint32_t cand = 0u;
#pragma unroll
      for (int t = 0; t < 16; ++t) cand |= (screen(t >> 2, t & 3) < etol ? 1u : 0u) << t;
      cand &= mask;
      while (cand) {
        const int t = __ffs(cand) - 1;
        cand &= cand - 1u;
        const int a = t >> 2, c = t & 3;
        const float d2 = dist2(-0.5f * pick(XR, a), -0.5f * pick(YR, a), -0.5f * pick(ZR, a),
                               pick(X, c), pick(Y, c), pick(Z, c));
        const float dd = sqrtf(d2) - (pick(RR, a) + pick(Rc, c));
        const int slot = 16 * (e.y & 0xFFFF) + t;  // row of blk_pidx: resolved at the end
        if (dd < best) {
          best = dd;
          bidx = slot;
        } else if (dd == best && bidx != INT_MAX &&
                   __ldg(r.blk_pidx + slot) < __ldg(r.blk_pidx + bidx)) {
          bidx = slot;  // exact tie: the smaller pair index wins
        }
      }
      set_row();
    }
    if (BITS && mask) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if ((mask >> (4 * a + c)) & 1u) {
            const float d2 = dist2(-0.5f * xr4[a], -0.5f * yr4[a], -0.5f * zr4[a], xj[c], yj[c],
                                   zj[c]);
            if (sqrtf(d2) - (pick(RR, a) + rj[c]) < 0.0f) {
              const int pidx = __ldg(r.blk_pidx + 16 * (e.y & 0xFFFF) + 4 * a + c);
              atomicOr(bm + (pidx >> 5), 1u << (pidx & 31));
            }
          }
        }
    }
    if (rr & 1) {  // group-wide best, every two rounds
      gbest = fminf(gbest, fkey_inv(__reduce_min_sync(0xffffffffu, fkey(best))));
      set_row();
    }
  }
  bidx = bidx == INT_MAX ? INT_MAX : __ldg(r.blk_pidx + bidx);  // slot -> pair index
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
    if (ob < best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  if (lane == 0 && A.dmin) {
    const bool none = bidx == INT_MAX;
    A.dmin[b] = none ? __int_as_float(0x7f800000) : best;
    A.worst[b] = none ? -1 : bidx;
    if (A.wdiff) pair_diff(r, A, b, none ? -1 : bidx, xc, yc, zc);
  }
  if (BITS) {
    __syncwarp();
    for (int w = lane; w < W; w += 32) A.bits[b * (int64_t)W + w] = bm[w];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The same map-reduce with whole blocks culled by group bounding spheres.
//
// Every 4-sphere group gets a bounding sphere (C_g, R_g): for a group on one
// link, a host-made sphere in that link's frame moved with the link;
// otherwise the mean of its centres and the largest |c - C_g| + r; both
// widened for float rounding.  For any
// pair (a in group i, b in group j), d_ab >= |C_i - C_j| - R_i - R_j =: lb, so
// a block whose lb exceeds an upper bound on d_min holds no candidate for the
// minimum (nor, with lb >= 0, a colliding pair).  Pass 1 finds the block of
// smallest lb and the exact minimum of its pairs, a real pair distance and
// so an upper bound on d_min, and keeps every block's lb as a half, rounded
// down below a margin for the approximate square root; pass 2 walks the
// schedule again, keeps the blocks whose stored lb is within the margin of
// the current bound (or below 0 when the pair bits are wanted) -- a superset
// of the blocks an exact test would keep -- queues them warp-wide (ballot +
// prefix count) and screens 32 queued blocks at a time with the usual screen
// and exact path.  The culled path forms the row copies of a block's spheres
// (-2 c) when it screens the block, and keeps the bounds where the full
// map-reduce keeps those copies.  The result -- d_min, the worst pair with its tie rule, the bits --
// is that of the full map-reduce; only blocks that cannot affect it are
// skipped.
template <bool FULL, bool BITS>
__device__ __forceinline__ void pair_one_culled(const DevRobot& r, const PairSchedule32& ps,
                                                const FwdArgs& A, int64_t b, float* ws,
                                                const float4* radw, int lane) {
  const PairPlan pl(r.n, r.Sg, r.P, BITS);
  float* xr = ws + pl.xr;
  float* xc = ws + pl.xc;
  float* yc = ws + pl.yc;
  float* zc = ws + pl.zc;
  float* nn = ws + pl.nn;
  float4* gb = reinterpret_cast<float4*>(ws + pl.gb);
  uint32_t* qu = reinterpret_cast<uint32_t*>(ws + pl.q);
  uint32_t* bm = reinterpret_cast<uint32_t*>(ws + pl.bits);
  const char* cxc = reinterpret_cast<const char*>(xc);
  const char* cyc = reinterpret_cast<const char*>(yc);
  const char* czc = reinterpret_cast<const char*>(zc);
  const char* cnn = reinterpret_cast<const char*>(nn);
  const char* crad = reinterpret_cast<const char*>(radw);
  const int n = r.n, S = r.S, Sg = r.Sg;
  const int W = (r.P + 31) >> 5;
  const float margin = r.margin, etol = r.etol, nrmin = -r.rmin;
  const int rounds = ps.rounds;
  // ---- stage the link poses (contiguous), then place the spheres ----
  {
    // asynchronous copies straight into shared memory (no register round
    // trip; with pass 1's schedule entries loaded a round ahead: humanoid48
    // pair stage 0.1238 -> 0.1193 ms)
    const float4* src = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
    float4* dst = reinterpret_cast<float4*>(xr);
    for (int i = lane; i < 3 * n; i += 32) {
      const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(dst + i));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(src + i));
    }
    asm volatile("cp.async.commit_group;");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  __syncwarp();
  if (r.sph_vec4) {
    // Every group of 4 spheres lies on one link: one lane a group reads the
    // link's pose once, places the 4 centres (the same arithmetic as the
    // per-sphere loop below), stores them as one float4 of each SoA array,
    // writes the group's 12 output floats as three float4 and forms the
    // group's bounding sphere from the same pose (humanoid48 pair stage
    // 0.1517 -> 0.1443 ms against the per-sphere loop, the same bits).
    float* so = A.sph ? A.sph + b * (int64_t)S * 3 : nullptr;
    const bool so4 = so != nullptr && (reinterpret_cast<uintptr_t>(so) & 15u) == 0;
    for (int g = lane; g < Sg; g += 32) {
      const int gl = __ldg(r.grp_link + g);
      const float4* T4 = reinterpret_cast<const float4*>(xr) + 3 * gl;  // the staged pose
      const float4 t0 = T4[0], t1 = T4[1], t2 = T4[2];
      const float T[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
      float cx[4], cy[4], cz[4], nv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 sp = __ldg(r.sph + 4 * g + q);
        const float cl[3] = {sp.x, sp.y, sp.z};
        float c[3];
        rot(T, cl, c);
        cx[q] = c[0] + T[9];
        cy[q] = c[1] + T[10];
        cz[q] = c[2] + T[11];
        nv[q] = fmaf(-sp.w, sp.w, fmaf(cz[q], cz[q], fmaf(cy[q], cy[q], cx[q] * cx[q])));
      }
      reinterpret_cast<float4*>(xc)[g] = make_float4(cx[0], cx[1], cx[2], cx[3]);
      reinterpret_cast<float4*>(yc)[g] = make_float4(cy[0], cy[1], cy[2], cy[3]);
      reinterpret_cast<float4*>(zc)[g] = make_float4(cz[0], cz[1], cz[2], cz[3]);
      reinterpret_cast<float4*>(nn)[g] = make_float4(nv[0], nv[1], nv[2], nv[3]);
      if (so) {
        const float o[12] = {cx[0], cy[0], cz[0], cx[1], cy[1], cz[1],
                             cx[2], cy[2], cz[2], cx[3], cy[3], cz[3]};
        float* og = so + 12 * g;
        if (so4) {
          float4* o4 = reinterpret_cast<float4*>(og);
          o4[0] = make_float4(o[0], o[1], o[2], o[3]);
          o4[1] = make_float4(o[4], o[5], o[6], o[7]);
          o4[2] = make_float4(o[8], o[9], o[10], o[11]);
        } else {
#pragma unroll
          for (int q = 0; q < 12; ++q) og[q] = o[q];
        }
      }
      const float4 L = __ldg(r.grp_loc + g);
      const float cl[3] = {L.x, L.y, L.z};
      float c[3];
      rot(T, cl, c);
      const float scale = fabsf(T[9]) + fabsf(T[10]) + fabsf(T[11]) + fabsf(L.x) + fabsf(L.y) +
                          fabsf(L.z);
      gb[g] = make_float4(c[0] + T[9], c[1] + T[10], c[2] + T[11],
                          fmaf(scale, 1e-6f, fmaf(L.w, 1e-6f, L.w)) + 3e-6f);
    }
  } else {
    for (int s = lane; s < 4 * Sg; s += 32) {
      float c[3] = {0.0f, 0.0f, 0.0f};
      float rs = 0.0f;
      if (s < S) {
        const float4 sp = __ldg(r.sph + s);
        // the link's staged pose as three vector loads (48-byte rows)
        const float4* P4 = reinterpret_cast<const float4*>(xr) + 3 * __ldg(r.sph_link + s);
        const float4 p0 = P4[0], p1 = P4[1], p2 = P4[2];
        const float P[12] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w};
        const float cl[3] = {sp.x, sp.y, sp.z};
        rot(P, cl, c);
        c[0] += P[9];
        c[1] += P[10];
        c[2] += P[11];
        rs = sp.w;
        if (A.sph) {
          float* o = A.sph + (b * S + s) * 3;
          o[0] = c[0];
          o[1] = c[1];
          o[2] = c[2];
        }
      }
      xc[s] = c[0];
      yc[s] = c[1];
      zc[s] = c[2];
      nn[s] = fmaf(-rs, rs, fmaf(c[2], c[2], fmaf(c[1], c[1], c[0] * c[0])));  // |c|^2 - r^2
    }
    __syncwarp();
    for (int g = lane; g < Sg; g += 32) {  // group bounding spheres
      const int gl = __ldg(r.grp_link + g);
      if (gl >= 0) {  // one link: its host-made bound, moved with the link
        const float4 L = __ldg(r.grp_loc + g);
        const float4* T4 = reinterpret_cast<const float4*>(xr) + 3 * gl;  // the staged pose
        const float4 t0 = T4[0], t1 = T4[1], t2 = T4[2];
        const float T[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
        const float cl[3] = {L.x, L.y, L.z};
        float c[3];
        rot(T, cl, c);
        // widened for the rounding of this transform and of the sphere
        // placement (a few ulp of the coordinates' size each)
        const float scale = fabsf(T[9]) + fabsf(T[10]) + fabsf(T[11]) + fabsf(L.x) + fabsf(L.y) +
                            fabsf(L.z);
        gb[g] = make_float4(c[0] + T[9], c[1] + T[10], c[2] + T[11],
                            fmaf(scale, 1e-6f, fmaf(L.w, 1e-6f, L.w)) + 3e-6f);
        continue;
      }
      const int s0 = 4 * g, s1 = min(S, s0 + 4);
      float cx = 0.0f, cy = 0.0f, cz = 0.0f;
      for (int s = s0; s < s1; ++s) {
        cx += xc[s];
        cy += yc[s];
        cz += zc[s];
      }
      const float inv = 1.0f / (float)max(s1 - s0, 1);
      cx *= inv;
      cy *= inv;
      cz *= inv;
      const float4 rad = radw[g];
      float R = 0.0f;
      for (int s = s0; s < s1; ++s)
        R = fmaxf(R, sqrtf(dist2(cx, cy, cz, xc[s], yc[s], zc[s])) + pick(rad, s - s0));
      gb[g] = make_float4(cx, cy, cz, fmaf(R, 1e-6f, R) + 3e-6f);  // widened for rounding
    }
  }
  if (BITS)
    for (int w = lane; w < W; w += 32) bm[w] = 0u;
  __syncwarp();
  if (!A.dmin && !BITS) return;  // sphere placement only
  if (rounds == 0) {
    if (lane == 0 && A.dmin) {
      A.dmin[b] = __int_as_float(0x7f800000);
      A.worst[b] = -1;
      if (A.wdiff) pair_diff(r, A, b, -1, xc, yc, zc);
    }
    if (BITS)
      for (int w = lane; w < W; w += 32) A.bits[b * (int64_t)W + w] = 0u;
    return;
  }
  const float inf = __int_as_float(0x7f800000);
  // ---- pass 1: the block of smallest lower bound (approximately: any block
  // gives a valid bound), and the exact minimum of its pairs ----
  // The lower bounds are kept for pass 2 as halves in the (now free) row
  // region when they fit, rounded down after a widening that covers the
  // approximate square root, so that pass 2 keeps every block its exact test
  // would keep (and at most a few more, within the half's rounding).
  const bool keep_lb = rounds * 32 <= 2 * pl.ra_words();
  __half* lb16 = reinterpret_cast<__half*>(xr);
  // the schedule's byte offsets of a block's two groups in the per-warp
  // sphere arrays (16 bytes a group) are also their offsets in gb
  const char* cgb = reinterpret_cast<const char*>(gb);
  float lbmin = inf;
  int rbest = 0;  // the round of the lane's smallest bound (its entry is
                  // reloaded once at the end: 0.1408 -> 0.1375 ms on humanoid48)
  uint2 en = __ldg(ps.ent + lane);  // one round ahead (the schedule ends with a null round)
  for (int rr = 0; rr < rounds; ++rr) {
    const uint2 e = en;
    en = __ldg(ps.ent + (rr + 1) * 32 + lane);
    __half low = __float2half(inf);  // null entries are never kept
    if ((e.y >> 16) != 0u) {  // a real block
      const float4 P4 = lds4(cgb, e.x & 0xFFFF), Q4 = lds4(cgb, e.x >> 16);
      const float D2 = fmaxf(dist2(P4.x, P4.y, P4.z, Q4.x, Q4.y, Q4.z), 1e-30f);
      const float dist = D2 * rsqrtf(D2);  // approximate square root
      // the lower bound widened for the approximate square root: 4e-6 of
      // the distance here, 2 x 2e-6 in the group radii
      const float lb = fmaf(dist, 0.999996f, -(P4.w + Q4.w));
      if (lb < lbmin) {
        lbmin = lb;
        rbest = rr;
      }
      low = __float2half_rd(lb);
    }
    if (keep_lb) lb16[rr * 32 + lane] = low;
  }
  float gbest;
  {
    const int kmin = __reduce_min_sync(0xffffffffu, fkey(lbmin));
    const int src = __ffs(__ballot_sync(0xffffffffu, fkey(lbmin) == kmin)) - 1;
    const uint2 e = __ldg(ps.ent + __shfl_sync(0xffffffffu, rbest, src) * 32 + src);
    float d = inf;
    const int t = lane & 15, a = t >> 2, c = t & 3;
    if (lane < 16 && ((e.y >> 16) >> t) & 1u) {
      const uint32_t ro = e.x & 0xFFFF, co = e.x >> 16;
      const float* pi = reinterpret_cast<const float*>(cxc + ro);
      const float* pyi = reinterpret_cast<const float*>(cyc + ro);
      const float* pzi = reinterpret_cast<const float*>(czc + ro);
      const float* pj = reinterpret_cast<const float*>(cxc + co);
      const float* pyj = reinterpret_cast<const float*>(cyc + co);
      const float* pzj = reinterpret_cast<const float*>(czc + co);
      d = sqrtf(dist2(pi[a], pyi[a], pzi[a], pj[c], pyj[c], pzj[c])) -
          (pick(lds4(crad, ro), a) + pick(lds4(crad, co), c));
    }
    gbest = fkey_inv(__reduce_min_sync(0xffffffffu, fkey(d)));  // a real pair: d_min <= gbest
  }
  // ---- pass 2: queue the surviving blocks, screen 32 at a time ----
  float best = 1e15f;
  int bidx = INT_MAX;
  int qn = 0;  // warp-uniform queue length
  // a block survives when its lower bound is within the screen's reach of
  // the current bound (or below zero when every colliding pair is wanted)
  const float reach_tol = 2.0f * margin;
  // the survival threshold changes only at a drain (hoisted out of the
  // per-round test: humanoid48 pair stage 0.1517 -> 0.1477 ms)
  float thr = fminf(best, gbest) + reach_tol;
  auto screen_block = [&](uint2 e) {
    const uint32_t ro = e.x & 0xFFFF, co = e.x >> 16;
    const uint32_t mask = e.y >> 16;
    const float4 XC = lds4(cxc, ro), YC = lds4(cyc, ro), ZC = lds4(czc, ro);
    const float4 XR = make_float4(-2.0f * XC.x, -2.0f * XC.y, -2.0f * XC.z, -2.0f * XC.w);
    const float4 YR = make_float4(-2.0f * YC.x, -2.0f * YC.y, -2.0f * YC.z, -2.0f * YC.w);
    const float4 ZR = make_float4(-2.0f * ZC.x, -2.0f * ZC.y, -2.0f * ZC.z, -2.0f * ZC.w);
    const float4 RR = lds4(crad, ro), NI = lds4(cnn, ro);
    const float4 CC = make_float4(fmaf(RR.x, RR.x, NI.x), fmaf(RR.y, RR.y, NI.y),
                                  fmaf(RR.z, RR.z, NI.z), fmaf(RR.w, RR.w, NI.w));  // |c_i|^2
    const float bb = fminf(best, gbest) + margin;
    const float T[4] = {fmaxf(bb + RR.x, nrmin), fmaxf(bb + RR.y, nrmin),
                        fmaxf(bb + RR.z, nrmin), fmaxf(bb + RR.w, nrmin)};
    const float C4[4] = {CC.x, CC.y, CC.z, CC.w};
    const float xr4[4] = {XR.x, XR.y, XR.z, XR.w}, yr4[4] = {YR.x, YR.y, YR.z, YR.w},
                zr4[4] = {ZR.x, ZR.y, ZR.z, ZR.w};
    const float4 X = lds4(cxc, co), Y = lds4(cyc, co), Z = lds4(czc, co), N = lds4(cnn, co),
                 Rc = lds4(crad, co);
    const float xj[4] = {X.x, X.y, X.z, X.w}, yj[4] = {Y.x, Y.y, Y.z, Y.w},
                zj[4] = {Z.x, Z.y, Z.z, Z.w}, nj[4] = {N.x, N.y, N.z, N.w},
                rj[4] = {Rc.x, Rc.y, Rc.z, Rc.w};
    auto screen = [&](int a, int c) {
      const float Ai = fmaf(-T[a], T[a], C4[a]);
      return fmaf(-2.0f * T[a], rj[c],
                  fmaf(zr4[a], zj[c], fmaf(yr4[a], yj[c], fmaf(xr4[a], xj[c], Ai + nj[c]))));
    };
    uint32_t cand = 0u;
#pragma unroll
    for (int t = 0; t < 16; ++t) cand |= (screen(t >> 2, t & 3) < etol ? 1u : 0u) << t;
    cand &= mask;
    while (cand) {
      const int t = __ffs(cand) - 1;
      cand &= cand - 1u;
      const int a = t >> 2, c = t & 3;
      // the candidate's centres and radii from shared memory (a dynamic index
      // into the register copies would put those in local memory)
      const float d2 = dist2(reinterpret_cast<const float*>(cxc + ro)[a],
                             reinterpret_cast<const float*>(cyc + ro)[a],
                             reinterpret_cast<const float*>(czc + ro)[a],
                             reinterpret_cast<const float*>(cxc + co)[c],
                             reinterpret_cast<const float*>(cyc + co)[c],
                             reinterpret_cast<const float*>(czc + co)[c]);
      const float dd = sqrtf(d2) - (reinterpret_cast<const float*>(crad + ro)[a] +
                                    reinterpret_cast<const float*>(crad + co)[c]);
      const int slot = 16 * (e.y & 0xFFFF) + t;  // row of blk_pidx: resolved at the end
      if (dd < best) {
        best = dd;
        bidx = slot;
      } else if (dd == best && bidx != INT_MAX &&
                 __ldg(r.blk_pidx + slot) < __ldg(r.blk_pidx + bidx)) {
        bidx = slot;  // exact tie: the smaller pair index wins
      }
    }
    if (BITS && mask) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if ((mask >> (4 * a + c)) & 1u) {
            const float d2 = dist2(-0.5f * xr4[a], -0.5f * yr4[a], -0.5f * zr4[a], xj[c], yj[c],
                                   zj[c]);
            if (sqrtf(d2) - (pick(RR, a) + rj[c]) < 0.0f) {
              const int pidx = __ldg(r.blk_pidx + 16 * (e.y & 0xFFFF) + 4 * a + c);
              atomicOr(bm + (pidx >> 5), 1u << (pidx & 31));
            }
          }
        }
    }
  };
  auto drain = [&](int count) {  // screen queue entries [0, count), one per lane
    const uint2 e = lane < count ? __ldg(ps.ent + qu[lane]) : make_uint2(0u, 0u);
    __syncwarp();
    if ((e.y >> 16) != 0u) screen_block(e);
    gbest = fminf(gbest, fkey_inv(__reduce_min_sync(0xffffffffu, fkey(best))));
  };
  if (keep_lb) {
    // Per chunk of 32 rounds, each lane first marks its surviving blocks in a
    // bit mask (one half load and one compare a round), then the survivors are
    // queued in lane order, positions from a warp scan of the lanes' counts,
    // and screened 32 at a time.  The threshold is refreshed per chunk; the
    // order of the screening does not change the result (the exact path keeps
    // the lexicographic (d, index) minimum).  Against a per-round ballot and
    // queue update: humanoid48 pair stage 0.1372 -> 0.1253 ms, same bits.
    for (int r0 = 0; r0 < rounds; r0 += 32) {
      const int r1 = min(rounds, r0 + 32);
      const float th = fminf(best, gbest) + reach_tol;
      uint32_t km = 0u;
      for (int rr = r0; rr < r1; ++rr) {  // null entries hold +inf
        const float lbv = __half2float(lb16[rr * 32 + lane]);
        km |= (lbv <= th || (BITS && lbv <= reach_tol) ? 1u : 0u) << (rr - r0);
      }
      const int cnt = __popc(km);
      int off = cnt;  // inclusive scan of the counts over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      const int tot = __shfl_sync(0xffffffffu, off, 31);
      int pos = off - cnt;
      for (int w0 = 0; w0 < tot; w0 += 32) {
        while (km && pos < w0 + 32) {
          const int rr = r0 + __ffs(km) - 1;
          km &= km - 1u;
          qu[pos - w0] = (uint32_t)(rr * 32 + lane);
          ++pos;
        }
        __syncwarp();
        drain(min(32, tot - w0));
        __syncwarp();
      }
    }
  } else {
    for (int rr = 0; rr < rounds; ++rr) {
      const int idx = rr * 32 + lane;
      // lb <= bound + tol  <=>  |C_i - C_j| <= t := bound + tol + R_i + R_j,
      // tested on squares (t >= 0); the tolerance covers the float rounding
      bool keep = false;
      if (keep_lb) {  // null entries hold +inf
        const float lbv = __half2float(lb16[idx]);
        keep = lbv <= thr || (BITS && lbv <= reach_tol);
      } else {
        const uint2 e = __ldg(ps.ent + idx);
        if ((e.y >> 16) != 0u) {
          const float4 P4 = gb[(e.x & 0xFFFF) >> 4], Q4 = gb[(e.x >> 16) >> 4];
          const float D2 = dist2(P4.x, P4.y, P4.z, Q4.x, Q4.y, Q4.z);
          const float RR2 = P4.w + Q4.w + reach_tol;
          const float t = fminf(best, gbest) + RR2;
          keep = (t >= 0.0f && D2 <= t * t) || (BITS && RR2 >= 0.0f && D2 <= RR2 * RR2);
        }
      }
      const uint32_t ball = __ballot_sync(0xffffffffu, keep);
      if (keep) qu[qn + __popc(ball & ((1u << lane) - 1u))] = (uint32_t)idx;
      qn += __popc(ball);
      if (qn >= 32) {
        __syncwarp();
        drain(32);
        thr = fminf(best, gbest) + reach_tol;
        __syncwarp();
        const uint32_t moved = lane + 32 < qn ? qu[lane + 32] : 0u;  // at most 31 left
        __syncwarp();
        if (lane + 32 < qn) qu[lane] = moved;
        qn -= 32;
        __syncwarp();
      }
    }
    __syncwarp();
    if (qn > 0) drain(qn);
  }
  bidx = bidx == INT_MAX ? INT_MAX : __ldg(r.blk_pidx + bidx);  // slot -> pair index
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
    if (ob < best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  if (lane == 0 && A.dmin) {
    const bool none = bidx == INT_MAX;
    A.dmin[b] = none ? __int_as_float(0x7f800000) : best;
    A.worst[b] = none ? -1 : bidx;
    if (A.wdiff) pair_diff(r, A, b, none ? -1 : bidx, xc, yc, zc);
  }
  if (BITS) {
    __syncwarp();
    for (int w = lane; w < W; w += 32) A.bits[b * (int64_t)W + w] = bm[w];
  }
  __syncwarp();
}

}  // namespace wbe
