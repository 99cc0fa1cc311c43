// k_pair.cu -- sphere placement and the self-collision map-reduce (Sec. 6.2),
// one warp per configuration.
//
// A warp reads its configuration's world link poses (config-major, written by
// the tree kernel), places the spheres (c_s = R_l c_local + p_l, Sec. 6.1.1)
// into shared memory as four SoA arrays (x, y, z, |c|^2) and writes the
// sphere output.  The pair blocks (4x4 sphere groups, dealt by the host so
// that the 8 lanes of a shared-memory phase read distinct bank groups, rows
// kept per lane in runs) are then screened with
//   e = |c_i|^2 + |c_j|^2 - 2 c_i . c_j - t^2,
//   t = max(best + r_i + margin, -r_min) + r_j >= 0,
// which is negative exactly when |c_i - c_j| < t.  Raising the row term to
// -r_min only widens the screen, and keeps t >= 0 so that t^2 is monotone.
// best is the warp-wide running minimum, refreshed every two rounds with one
// integer min-reduction over an order-preserving key, so the exact path --
// sqrt distance, pair index, lexicographic (d, index) compare -- only runs
// for screened-in pairs, one candidate at a time.  The screen fires on
// e < etol, a host bound on the float rounding of the expanded form, so it
// never drops a pair the exact path would keep.  A 5-step shuffle reduction
// of (d, index) finishes the configuration: one configuration never spans
// more than one warp, so the paper's second reduce kernel becomes a register
// reduction.
#include "spatial.cuh"

#include <climits>

namespace wbe {

__host__ __device__ constexpr int a32(int x) { return (x + 31) & ~31; }

struct PairPlan {  // per warp, 32-bit words
  int sx, sy, sz, sc, bits, total;
  __host__ __device__ PairPlan(int Sg, int P, bool with_bits) {
    const int m = a32(4 * Sg);
    sx = 0;
    sy = m;
    sz = 2 * m;
    sc = 3 * m;
    bits = 4 * m;
    total = bits + (with_bits ? a32((P + 31) / 32) : 0);
  }
};

size_t pair_smem(const DevRobot& r, int warps, bool bits) {
  return sizeof(float) * ((size_t)a32(4 * r.Sg) + (size_t)warps * PairPlan(r.Sg, r.P, bits).total);
}

// order-preserving map of a float to a signed int (and back)
__device__ __forceinline__ int fkey(float f) {
  const int i = __float_as_int(f);
  return i < 0 ? i ^ 0x7FFFFFFF : i;
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k < 0 ? k ^ 0x7FFFFFFF : k); }

template <bool FULL, bool BITS>
__global__ void __launch_bounds__(256, 3) pair_kernel(DevRobot r, PairSchedule ps, FwdArgs A) {
  extern __shared__ __align__(128) float smem[];
  const PairPlan pl(r.Sg, r.P, BITS);
  float4* rad = reinterpret_cast<float4*>(smem);
  for (int i = threadIdx.x; i < r.Sg; i += blockDim.x) rad[i] = __ldg(r.grp_rad + i);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  float* ws = smem + a32(4 * r.Sg) + warp * pl.total;
  float* sx = ws + pl.sx;
  float* sy = ws + pl.sy;
  float* sz = ws + pl.sz;
  float* sc = ws + pl.sc;
  uint32_t* bm = reinterpret_cast<uint32_t*>(ws + pl.bits);
  const float4* sx4 = reinterpret_cast<const float4*>(sx);
  const float4* sy4 = reinterpret_cast<const float4*>(sy);
  const float4* sz4 = reinterpret_cast<const float4*>(sz);
  const float4* sc4 = reinterpret_cast<const float4*>(sc);
  const int n = r.n, S = r.S;
  const int W = (r.P + 31) >> 5;
  const float margin = r.margin, etol = r.etol, nrmin = -r.rmin;
  const int rounds = ps.rounds;

  for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < A.B; b += (int64_t)gridDim.x * wpb) {
    // ---- sphere centres from the link poses ----
    const float* pose = A.pose + b * (int64_t)n * 12;
    for (int s = lane; s < 4 * r.Sg; s += 32) {
      float c[3] = {0.0f, 0.0f, 0.0f};
      if (s < S) {
        const float4 sp = __ldg(r.sph + s);
        const int l = __ldg(r.sph_link + s);
        const float4* P4 = reinterpret_cast<const float4*>(pose + 12 * l);
        const float4 p0 = P4[0], p1 = P4[1], p2 = P4[2];
        const float R[9] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x};
        const float cl[3] = {sp.x, sp.y, sp.z};
        rot(R, cl, c);
        c[0] += p2.y;
        c[1] += p2.z;
        c[2] += p2.w;
        if (A.sph) {
          float* o = A.sph + (b * S + s) * 3;
          o[0] = c[0];
          o[1] = c[1];
          o[2] = c[2];
        }
      }
      sx[s] = c[0];
      sy[s] = c[1];
      sz[s] = c[2];
      sc[s] = fmaf(c[2], c[2], fmaf(c[1], c[1], c[0] * c[0]));
    }
    if (BITS)
      for (int w = lane; w < W; w += 32) bm[w] = 0u;
    __syncwarp();
    if (!A.dmin && !BITS) {  // sphere placement only
      __syncwarp();
      continue;
    }
    if (rounds == 0) {
      if (lane == 0 && A.dmin) {
        A.dmin[b] = __int_as_float(0x7f800000);
        A.worst[b] = -1;
      }
      if (BITS)
        for (int w = lane; w < W; w += 32) A.bits[b * (int64_t)W + w] = 0u;
      continue;
    }
    float best = 1e15f;
    int bidx = INT_MAX;
    uint2 nxt = __ldg(ps.ent + lane);
    // seed: the exact distance of one pair of the lane's first block
    if (FULL && (nxt.x >> 16) != 0u) {
      const int gi = nxt.x & 0xFF, gj = (nxt.x >> 8) & 0xFF;
      const float d2 = dist2(sx[4 * gi], sy[4 * gi], sz[4 * gi], sx[4 * gj], sy[4 * gj], sz[4 * gj]);
      best = sqrtf(d2) - (rad[gi].x + rad[gj].x);
      bidx = __ldg(r.blk_pidx + 16 * nxt.y);
    }
    float gbest = fkey_inv(__reduce_min_sync(0xffffffffu, fkey(best)));
    int cur = -1;
    float xi2[4], yi2[4], zi2[4], cci[4], Ti[4];
    auto set_row = [&]() {
      const float bb = fminf(best, gbest) + margin;
      const float4 Rr = rad[cur];
      Ti[0] = fmaxf(bb + Rr.x, nrmin);
      Ti[1] = fmaxf(bb + Rr.y, nrmin);
      Ti[2] = fmaxf(bb + Rr.z, nrmin);
      Ti[3] = fmaxf(bb + Rr.w, nrmin);
    };
    for (int rr = 0; rr < rounds; ++rr) {
      const uint2 e = nxt;
      nxt = __ldg(ps.ent + (rr + 1) * 32 + lane);  // the schedule has a null round at the end
      const uint32_t mask = e.x >> 16;
      const int gi = e.x & 0xFF, gj = (e.x >> 8) & 0xFF;
      if (gi != cur) {
        cur = gi;
        const float4 X = sx4[gi], Y = sy4[gi], Z = sz4[gi], C = sc4[gi];
        xi2[0] = -2.0f * X.x; xi2[1] = -2.0f * X.y; xi2[2] = -2.0f * X.z; xi2[3] = -2.0f * X.w;
        yi2[0] = -2.0f * Y.x; yi2[1] = -2.0f * Y.y; yi2[2] = -2.0f * Y.z; yi2[3] = -2.0f * Y.w;
        zi2[0] = -2.0f * Z.x; zi2[1] = -2.0f * Z.y; zi2[2] = -2.0f * Z.z; zi2[3] = -2.0f * Z.w;
        cci[0] = C.x; cci[1] = C.y; cci[2] = C.z; cci[3] = C.w;
        set_row();
      }
      const float4 X = sx4[gj], Y = sy4[gj], Z = sz4[gj], C = sc4[gj], Rr = rad[gj];
      const float xj[4] = {X.x, X.y, X.z, X.w};
      const float yj[4] = {Y.x, Y.y, Y.z, Y.w};
      const float zj[4] = {Z.x, Z.y, Z.z, Z.w};
      const float ccj[4] = {C.x, C.y, C.z, C.w};
      const float rj[4] = {Rr.x, Rr.y, Rr.z, Rr.w};
      auto screen = [&](int a, int c) {
        const float t = Ti[a] + rj[c];
        return fmaf(-t, t, fmaf(zi2[a], zj[c], fmaf(yi2[a], yj[c], fmaf(xi2[a], xj[c], cci[a] + ccj[c]))));
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
        const float4 Ri = rad[cur];
        while (cand) {
          const int t = __ffs(cand) - 1;
          cand &= cand - 1u;
          const int a = t >> 2, c = t & 3;
          const float xa = (a == 0 ? xi2[0] : a == 1 ? xi2[1] : a == 2 ? xi2[2] : xi2[3]);
          const float ya = (a == 0 ? yi2[0] : a == 1 ? yi2[1] : a == 2 ? yi2[2] : yi2[3]);
          const float za = (a == 0 ? zi2[0] : a == 1 ? zi2[1] : a == 2 ? zi2[2] : zi2[3]);
          const float ra = (a == 0 ? Ri.x : a == 1 ? Ri.y : a == 2 ? Ri.z : Ri.w);
          const float xc = (c == 0 ? X.x : c == 1 ? X.y : c == 2 ? X.z : X.w);
          const float yc = (c == 0 ? Y.x : c == 1 ? Y.y : c == 2 ? Y.z : Y.w);
          const float zc = (c == 0 ? Z.x : c == 1 ? Z.y : c == 2 ? Z.z : Z.w);
          const float rc = (c == 0 ? Rr.x : c == 1 ? Rr.y : c == 2 ? Rr.z : Rr.w);
          const float d2 = dist2(-0.5f * xa, -0.5f * ya, -0.5f * za, xc, yc, zc);
          const float dd = sqrtf(d2) - (ra + rc);
          if (dd <= best) {
            const int pidx = __ldg(r.blk_pidx + 16 * e.y + t);
            if (dd < best || pidx < bidx) {
              best = dd;
              bidx = pidx;
            }
          }
        }
        set_row();
      }
      if (BITS && mask) {
        const float4 Ri = rad[cur];
        const float ri[4] = {Ri.x, Ri.y, Ri.z, Ri.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if ((mask >> (4 * a + c)) & 1u) {
              const float d2 =
                  dist2(-0.5f * xi2[a], -0.5f * yi2[a], -0.5f * zi2[a], xj[c], yj[c], zj[c]);
              if (sqrtf(d2) - (ri[a] + rj[c]) < 0.0f) {
                const int pidx = __ldg(r.blk_pidx + 16 * e.y + 4 * a + c);
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
    }
    if (BITS) {
      __syncwarp();
      for (int w = lane; w < W; w += 32) A.bits[b * (int64_t)W + w] = bm[w];
    }
    __syncwarp();
  }
}

template <bool FULL, bool BITS>
static cudaError_t pair_launch_t(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                                 int grid, int warps, size_t smem, cudaStream_t s, int* occ) {
  auto kern = pair_kernel<FULL, BITS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, warps * 32, smem);
  kern<<<grid, warps * 32, smem, s>>>(r, ps, a);
  return cudaGetLastError();
}

static cudaError_t pair_dispatch(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                                 int grid, int warps, cudaStream_t s, int* occ) {
  const bool bits = a.bits != nullptr;
  const size_t smem = pair_smem(r, warps, bits);
  if (r.all_full) {
    return bits ? pair_launch_t<true, true>(r, ps, a, grid, warps, smem, s, occ)
                : pair_launch_t<true, false>(r, ps, a, grid, warps, smem, s, occ);
  }
  return bits ? pair_launch_t<false, true>(r, ps, a, grid, warps, smem, s, occ)
              : pair_launch_t<false, false>(r, ps, a, grid, warps, smem, s, occ);
}

cudaError_t launch_pair(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a, int grid,
                        int warps, cudaStream_t s) {
  return pair_dispatch(r, ps, a, grid, warps, s, nullptr);
}

cudaError_t pair_max_blocks_per_sm(const DevRobot& r, int warps, bool bits, int* out) {
  FwdArgs a{};
  a.bits = bits ? reinterpret_cast<uint32_t*>(16) : nullptr;  // only selects the variant
  return pair_dispatch(r, PairSchedule{}, a, 0, warps, nullptr, out);
}

}  // namespace wbe
