// k_fused.cu -- fused whole-body kernels.
//
// Layout of the work: a CTA owns a tile of `cpb` consecutive configurations;
// each configuration is owned by a group of G lanes (G = 32: one warp per
// configuration; G < 32: 32/G configurations per warp).  Per tile:
//   1. the CTA stages q, qd, qdd (joint-major [d][B] in HBM) for its tile into
//      shared memory: each joint row of the tile is a contiguous run, loaded
//      coalesced;
//   2. each group runs its configuration through the stages, level by level
//      over the tree (Sec. 6.3 "tree-level parallelism"), synchronising with
//      __syncwarp (Tab. rnea_comparison "warp" sync), with link transforms,
//      sphere centres and dynamics state in shared memory;
//   3. the CTA writes the joint-major outputs of the tile back coalesced.
// The grid is persistent: CTAs loop over tiles with a grid stride.  Robot
// metadata that every level step needs (the level-ordered link table, axes,
// mimic factors, sphere-group radii) is copied to shared memory once per CTA.
//
// Pair stage (Sec. 6.2).  The host groups spheres in fours and the pair list
// into 4x4 group blocks, then deals the blocks to the G lanes so that, in
// every round, the 8 lanes of a shared-memory phase read distinct bank groups
// (block column gj = lane mod 8).  A lane keeps the 4 row spheres of its
// current block in registers and screens the 16 pairs of a block with the
// expanded squared form
//   e = (|c_i|^2 + |c_j|^2) - 2 c_i . c_j - t |t|,  t = best + r_i + margin + r_j,
// which is negative exactly when |c_i - c_j| < t (t <= 0 can never fire:
// the pair cannot beat best), at 6 float operations per pair.  `best` is the group-wide running minimum,
// refreshed by shuffles every four rounds, so only blocks that may hold a new
// minimum take the exact path: d = sqrt(|c_i - c_j|^2) - (r_i + r_j), pair
// index from the block table, (d, index) compared lexicographically.  The
// screen fires on e < etol, a host bound on the float rounding of the
// expanded form (128 ulp of (reach + r_max)^2), so it never drops a pair the
// exact path would keep.  The G lanes finally reduce (d, index) with
// shuffles: one configuration never spans more than one group, so the
// paper's second reduce kernel becomes a register reduction.
#include "spatial.cuh"

#include <climits>

namespace wbe {

__host__ __device__ constexpr int align32(int x) { return (x + 31) & ~31; }

// ---------------------------------------------------------------------------
// shared-memory plans (32-bit words), identical on host and device
// ---------------------------------------------------------------------------
struct CtaPlan {  // robot metadata cached per CTA
  int lvm, lev, rad, mm, ax, total;
  __host__ __device__ CtaPlan(int n, int nlev, int Sg) {
    int o = 0;
    lvm = o; o += align32(4 * n);
    lev = o; o += align32(nlev + 1);
    rad = o; o += align32(4 * Sg);
    mm = o;  o += align32(2 * n);
    ax = o;  o += align32(4 * n);
    total = o;
  }
};

struct FwdPlan {  // per configuration
  int q, q2, Rw, sx, sy, sz, sc, Rl, v, a, F, bits, total, stride;
  __host__ __device__ FwdPlan(int n, int d, int Sg, int P, bool with_bits) {
    int o = 0;
    q = o; o += align32(3 * d);    // q, qd, qdd of this tile (tau staged in q)
    q2 = o; o += align32(3 * d);   // the next tile's, loaded while this one runs
    const int u = o;
    // FK / pair phase
    Rw = u;
    sx = Rw + align32(12 * n);
    sy = sx + align32(4 * Sg);
    sz = sy + align32(4 * Sg);
    sc = sz + align32(4 * Sg);
    const int end1 = sc + align32(4 * Sg);
    // dynamics phase (aliases the FK / pair phase)
    Rl = u;
    v = Rl + align32(12 * n);
    a = v + align32(6 * n);
    F = a + align32(6 * n);
    const int end2 = F + align32(6 * n);
    o = end1 > end2 ? end1 : end2;
    bits = o;
    if (with_bits) o += align32((P + 31) / 32);
    total = o;
    stride = total + 4;  // +16 B: consecutive configurations start 4 banks apart
  }
};

struct BwdPlan {
  int q, q2, Rl, Rw, up, vb, lq, va, F, W, total, stride;
  __host__ __device__ BwdPlan(int n, int d) {
    int o = 0;
    q = o;  o += align32(4 * d);   // q, qd, qdd, g_tau  -> gq, gqd, gqdd
    q2 = o; o += align32(4 * d);   // the next tile's inputs
    Rl = o; o += align32(12 * n);
    Rw = o; o += align32(12 * n);  // later: up (6n) in the force sweep,
    up = Rw;                       //        vb (6n) + lq (3n) in the adjoint
    vb = Rw;
    lq = Rw + 6 * n;
    va = o; o += align32(12 * n);  // v (6n), a (6n)
    F = o;  o += align32(6 * n);
    W = o;  o += align32(6 * n);
    total = o;
    stride = total + 4;
  }
};

size_t fused_fwd_smem_per_config(const DevRobot& r, int G, bool bits) {
  (void)G;
  return sizeof(float) * (size_t)FwdPlan(r.n, r.d, r.Sg, r.P, bits).stride;
}
size_t fused_bwd_smem_per_config(const DevRobot& r, int G) {
  (void)G;
  return sizeof(float) * (size_t)BwdPlan(r.n, r.d).stride;
}
size_t fused_cta_smem(const DevRobot& r) {
  return sizeof(float) * (size_t)CtaPlan(r.n, r.nlev, r.Sg).total;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
struct Cta {
  const int4* lvm;
  const int* lev;
  const float4* rad;
  const float2* mm;
  const float4* ax;
};

__device__ __forceinline__ Cta load_cta(const DevRobot& r, float* smem) {
  const CtaPlan cp(r.n, r.nlev, r.Sg);
  int4* lvm = reinterpret_cast<int4*>(smem + cp.lvm);
  int* lev = reinterpret_cast<int*>(smem + cp.lev);
  float4* rad = reinterpret_cast<float4*>(smem + cp.rad);
  float2* mm = reinterpret_cast<float2*>(smem + cp.mm);
  float4* ax = reinterpret_cast<float4*>(smem + cp.ax);
  for (int i = threadIdx.x; i < r.n; i += blockDim.x) {
    lvm[i] = __ldg(r.lvm + i);
    mm[i] = __ldg(reinterpret_cast<const float2*>(r.mimic) + i);
    ax[i] = __ldg(reinterpret_cast<const float4*>(r.axis) + i);
  }
  for (int i = threadIdx.x; i <= r.nlev; i += blockDim.x) lev[i] = r.lev_start[i];
  for (int i = threadIdx.x; i < r.Sg; i += blockDim.x) rad[i] = __ldg(r.grp_rad + i);
  __syncthreads();
  return Cta{lvm, lev, rad, mm, ax};
}

__device__ __forceinline__ int meta_jidx(int z) { return (z & 0xFFFF) - 1; }
__device__ __forceinline__ int meta_jtype(int z) { return (z >> 16) & 0xFF; }
__device__ __forceinline__ bool meta_rotid(int z) { return ((z >> 24) & 0xFF) != 0; }

// Local transform (parent joint frame -> link frame) of link k = T_fixed *
// J(th): revolute R = R_f R_J(th) (Rodrigues), prismatic p = p_f + R_f a th.
__device__ __forceinline__ void local_tf(const DevRobot& r, int k, int jt, bool ident, float4 a,
                                         float th, float* out) {
  const float4* T4 = reinterpret_cast<const float4*>(r.Tf + 12 * k);
  const float4 t0 = __ldg(T4), t1 = __ldg(T4 + 1), t2 = __ldg(T4 + 2);
  const float Rf[9] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x};
  float p[3] = {t2.y, t2.z, t2.w};
  float R[9];
  if (jt == 1) {
    float s, c;
    sincosf(th, &s, &c);
    const float t = 1.0f - c;
    const float tx = t * a.x, ty = t * a.y, tz = t * a.z;
    const float sx = s * a.x, sy = s * a.y, sz = s * a.z;
    const float Rj[9] = {fmaf(tx, a.x, c),  fmaf(tx, a.y, -sz), fmaf(tx, a.z, sy),
                         fmaf(ty, a.x, sz), fmaf(ty, a.y, c),   fmaf(ty, a.z, -sx),
                         fmaf(tz, a.x, -sy), fmaf(tz, a.y, sx), fmaf(tz, a.z, c)};
    if (ident) {
#pragma unroll
      for (int e = 0; e < 9; ++e) R[e] = Rj[e];
    } else {
      matmul3(Rf, Rj, R);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e] = Rf[e];
    if (jt == 2) {
      const float s3[3] = {a.x * th, a.y * th, a.z * th};
      float Rs[3];
      rot(Rf, s3, Rs);
      p[0] += Rs[0];
      p[1] += Rs[1];
      p[2] += Rs[2];
    }
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) out[e] = R[e];
  out[9] = p[0];
  out[10] = p[1];
  out[11] = p[2];
}

// compose in place: W <- P o W  (W holds the local transform on entry)
__device__ __forceinline__ void compose_inplace(const float* P, float* W) {
  float L[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) L[e] = W[e];
  float R[9], t[3];
  matmul3(P, L, R);
  rot(P, L + 9, t);
#pragma unroll
  for (int e = 0; e < 9; ++e) W[e] = R[e];
  W[9] = P[9] + t[0];
  W[10] = P[10] + t[1];
  W[11] = P[11] + t[2];
}

__device__ __forceinline__ void load6(const float* s, float* d) {
#pragma unroll
  for (int e = 0; e < 6; ++e) d[e] = s[e];
}
__device__ __forceinline__ void store6(float* d, const float* s) {
#pragma unroll
  for (int e = 0; e < 6; ++e) d[e] = s[e];
}
__device__ __forceinline__ void load12(const float* s, float* d) {
#pragma unroll
  for (int e = 0; e < 12; ++e) d[e] = s[e];
}

template <int G>
__device__ __forceinline__ void group_min(float& best, int& idx) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ob < best || (ob == best && oi < idx)) {
      best = ob;
      idx = oi;
    }
  }
}

template <int G>
__device__ __forceinline__ float group_min_value(float v) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// Asynchronous copy of a tile's joint-major rows [d][B] into per-config
// shared arrays (cp.async: every load of the tile is in flight at once);
// missing configurations and NULL inputs read as zero.
__device__ __forceinline__ void cp_async_f32(float* sdst, const float* gsrc) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ void stage_rows(float* base, int stride, int dst_off, const float* src,
                                           int d, int64_t B, int64_t b0, int cpb) {
  for (int idx = threadIdx.x; idx < d * cpb; idx += blockDim.x) {
    const int j = idx / cpb, c = idx - j * cpb;
    const int64_t b = b0 + c;
    float* dst = base + c * stride + dst_off + j;
    if (src && b < B)
      cp_async_f32(dst, src + (int64_t)j * B + b);
    else
      *dst = 0.0f;
  }
}

__device__ __forceinline__ void unstage_rows(const float* base, int stride, int src_off,
                                             float* dst, int d, int64_t B, int64_t b0, int cpb) {
  for (int idx = threadIdx.x; idx < d * cpb; idx += blockDim.x) {
    const int j = idx / cpb, c = idx - j * cpb;
    const int64_t b = b0 + c;
    if (b < B) dst[(int64_t)j * B + b] = base[c * stride + src_off + j];
  }
}

// Local transforms of every link into T (parallel over links), then, if
// `world`, in-place composition level by level into world poses.
template <int G>
__device__ __forceinline__ void group_transforms(const DevRobot& r, const Cta& ct, int lig,
                                                 const float* qs, float* T, bool world) {
  for (int i = lig; i < r.n; i += G) {
    const int4 m = ct.lvm[i];
    const int k = m.x;
    const int j = meta_jidx(m.z);
    const float2 mm = ct.mm[k];
    const float th = j >= 0 ? fmaf(mm.x, qs[j], mm.y) : 0.0f;
    local_tf(r, k, meta_jtype(m.z), meta_rotid(m.z), ct.ax[k], th, T + 12 * k);
  }
  __syncwarp();
  if (!world) return;
  for (int lev = 1; lev < r.nlev; ++lev) {
    const int s1 = ct.lev[lev + 1];
    for (int i = ct.lev[lev] + lig; i < s1; i += G) {
      const int4 m = ct.lvm[i];
      float P[12];
      load12(T + 12 * m.y, P);
      compose_inplace(P, T + 12 * m.x);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(256, 3) fused_fwd_kernel(DevRobot r, PairSchedule ps, FwdArgs A,
                                                        int cpb) {
  extern __shared__ __align__(128) float smem[];
  const bool with_bits = A.bits != nullptr;
  const Cta ct = load_cta(r, smem);
  const FwdPlan pl(r.n, r.d, r.Sg, r.P, with_bits);
  float* base = smem + CtaPlan(r.n, r.nlev, r.Sg).total;
  const int lane = threadIdx.x & 31;
  const int lig = lane & (G - 1);
  const int cfg = threadIdx.x / G;  // configuration slot in the tile
  const int64_t B = A.B;
  const int64_t ntiles = (B + cpb - 1) / cpb;
  float* cs = base + (size_t)cfg * pl.stride;
  const int W = (r.P + 31) >> 5;
  const int n = r.n, d = r.d;

  auto stage = [&](int64_t t, int off) {
    const int64_t s0 = t * cpb;
    stage_rows(base, pl.stride, off, A.q, d, B, s0, cpb);
    stage_rows(base, pl.stride, off + d, A.qd, d, B, s0, cpb);
    stage_rows(base, pl.stride, off + 2 * d, A.qdd, d, B, s0, cpb);
    cp_async_commit();
  };
  if ((int64_t)blockIdx.x < ntiles) stage(blockIdx.x, pl.q);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t b0 = tile * cpb;
    const int qoff = (it & 1) ? pl.q2 : pl.q;
    cp_async_wait_all();
    __syncthreads();
    if (tile + gridDim.x < ntiles) stage(tile + gridDim.x, (it & 1) ? pl.q : pl.q2);
    const int64_t b = b0 + cfg;
    const bool live = b < B;
    float* qs = cs + qoff;
    // ---- forward kinematics: world poses in Rw ----
    float* Rw = cs + pl.Rw;
    group_transforms<G>(r, ct, lig, qs, Rw, true);
    // ---- sphere centres (SoA by component, padded to whole groups) ----
    float* sx = cs + pl.sx;
    float* sy = cs + pl.sy;
    float* sz = cs + pl.sz;
    float* sc = cs + pl.sc;
    for (int s = lig; s < 4 * r.Sg; s += G) {
      float c[3] = {0.0f, 0.0f, 0.0f};
      if (s < r.S) {
        const float4 sp = __ldg(r.sph + s);
        const int l = __ldg(r.sph_link + s);
        const float cl[3] = {sp.x, sp.y, sp.z};
        const float* P = Rw + 12 * l;
        rot(P, cl, c);
        c[0] += P[9];
        c[1] += P[10];
        c[2] += P[11];
      }
      sx[s] = c[0];
      sy[s] = c[1];
      sz[s] = c[2];
      sc[s] = fmaf(c[2], c[2], fmaf(c[1], c[1], c[0] * c[0]));
    }
    if (with_bits)
      for (int w = lig; w < W; w += G) reinterpret_cast<uint32_t*>(cs + pl.bits)[w] = 0u;
    __syncwarp();
    // ---- outputs: poses and sphere centres (config-major, contiguous) ----
    if (live && A.pose) {
      float4* dst = reinterpret_cast<float4*>(A.pose + b * (int64_t)n * 12);
      const float4* src = reinterpret_cast<const float4*>(Rw);
      for (int e = lig; e < 3 * n; e += G) dst[e] = src[e];
    }
    if (live && A.sph) {
      float* dst = A.sph + b * (int64_t)r.S * 3;
      for (int e = lig; e < 3 * r.S; e += G) {
        const int s = e / 3, c = e - 3 * s;
        dst[e] = (c == 0 ? sx : (c == 1 ? sy : sz))[s];
      }
    }
    // ---- self-collision: screened map over the lane's blocks, group reduce ----
    if (A.dmin || with_bits) {
      const float4* sx4 = reinterpret_cast<const float4*>(sx);
      const float4* sy4 = reinterpret_cast<const float4*>(sy);
      const float4* sz4 = reinterpret_cast<const float4*>(sz);
      const float4* sc4 = reinterpret_cast<const float4*>(sc);
      uint32_t* bm = reinterpret_cast<uint32_t*>(cs + pl.bits);
      const float BIG = 1e15f;
      float best = BIG, gbest = BIG;
      int bidx = INT_MAX;
      int cur = -1;
      float xi2[4], yi2[4], zi2[4], cci[4], Ti[4];
      const float margin = r.margin, etol = r.etol;
      // screen constants of the current row group: T_i = best + r_i + margin
      auto set_row = [&]() {
        const float bb = fminf(best, gbest);
        const float4 Rr = ct.rad[cur];
        Ti[0] = bb + Rr.x + margin;
        Ti[1] = bb + Rr.y + margin;
        Ti[2] = bb + Rr.z + margin;
        Ti[3] = bb + Rr.w + margin;
      };
      uint2 nxt = make_uint2(0u, 0u);
      if (ps.rounds > 0) nxt = __ldg(ps.ent + lig);
      for (int rr = 0; rr < ps.rounds; ++rr) {
        const uint2 e = nxt;
        if (rr + 1 < ps.rounds) nxt = __ldg(ps.ent + (rr + 1) * G + lig);
        const uint32_t mask = e.x >> 16;
        if (mask != 0u) {
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
          const float4 X = sx4[gj], Y = sy4[gj], Z = sz4[gj], C = sc4[gj], Rr = ct.rad[gj];
          const float xj[4] = {X.x, X.y, X.z, X.w};
          const float yj[4] = {Y.x, Y.y, Y.z, Y.w};
          const float zj[4] = {Z.x, Z.y, Z.z, Z.w};
          const float ccj[4] = {C.x, C.y, C.z, C.w};
          const float rj[4] = {Rr.x, Rr.y, Rr.z, Rr.w};
          // e(a, c) = |c_i - c_j|^2 - t |t|, t = T_i + r_j (t < 0 never fires)
          auto screen = [&](int a, int c) {
            const float t = Ti[a] + rj[c];
            return fmaf(-t, fabsf(t),
                        fmaf(zi2[a], zj[c], fmaf(yi2[a], yj[c], fmaf(xi2[a], xj[c], cci[a] + ccj[c]))));
          };
          float m;
          if (mask == 0xFFFFu) {
            float m4[4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
              m4[a] = fminf(fminf(screen(a, 0), screen(a, 1)), fminf(screen(a, 2), screen(a, 3)));
            m = fminf(fminf(m4[0], m4[1]), fminf(m4[2], m4[3]));
          } else {
            m = __int_as_float(0x7f800000);
#pragma unroll
            for (int t = 0; t < 16; ++t)
              if ((mask >> t) & 1u) m = fminf(m, screen(t >> 2, t & 3));
          }
          if (m < etol) {
            // exact path for the screened-in pairs (rare once best settles)
            const float4 Ri = ct.rad[cur];
            const float ri[4] = {Ri.x, Ri.y, Ri.z, Ri.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                if (((mask >> (4 * a + c)) & 1u) && screen(a, c) < etol) {
                  const float d2 = dist2(-0.5f * xi2[a], -0.5f * yi2[a], -0.5f * zi2[a], xj[c],
                                         yj[c], zj[c]);
                  const float dd = sqrtf(d2) - (ri[a] + rj[c]);
                  if (dd <= best) {
                    const int pidx = __ldg(r.blk_pidx + 16 * e.y + 4 * a + c);
                    if (dd < best || pidx < bidx) {
                      best = dd;
                      bidx = pidx;
                    }
                  }
                }
              }
            set_row();
          }
          if (with_bits) {
            const float4 Ri = ct.rad[cur];
            const float ri[4] = {Ri.x, Ri.y, Ri.z, Ri.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                if ((mask >> (4 * a + c)) & 1u) {
                  const float d2 = dist2(-0.5f * xi2[a], -0.5f * yi2[a], -0.5f * zi2[a], xj[c],
                                         yj[c], zj[c]);
                  if (sqrtf(d2) - (ri[a] + rj[c]) < 0.0f) {
                    const int pidx = __ldg(r.blk_pidx + 16 * e.y + 4 * a + c);
                    atomicOr(bm + (pidx >> 5), 1u << (pidx & 31));
                  }
                }
              }
          }
        }
        if (rr < 4 || (rr & 3) == 3) {  // refresh often while best is settling
          gbest = group_min_value<G>(best);
          if (cur >= 0) set_row();
        }
      }
      group_min<G>(best, bidx);
      if (live && lig == 0 && A.dmin) {
        const bool none = bidx == INT_MAX;
        A.dmin[b] = none ? __int_as_float(0x7f800000) : best;
        A.worst[b] = none ? -1 : bidx;
      }
      if (with_bits) {
        __syncwarp();
        if (live)
          for (int w = lig; w < W; w += G) A.bits[b * (int64_t)W + w] = bm[w];
      }
    }
    __syncwarp();
    // ---- RNEA (Alg. 4); local transforms recomputed (Rw / spheres are dead) ----
    if (A.tau) {
      float* Rl = cs + pl.Rl;
      float* v = cs + pl.v;
      float* a = cs + pl.a;
      float* F = cs + pl.F;
      const float* qd = qs + d;
      const float* qdd = qs + 2 * d;
      group_transforms<G>(r, ct, lig, qs, Rl, false);
      // pass 1, base -> tips: v, a
      for (int lev = 0; lev < r.nlev; ++lev) {
        const int s1 = ct.lev[lev + 1];
        for (int i = ct.lev[lev] + lig; i < s1; i += G) {
          const int4 m = ct.lvm[i];
          const int k = m.x, pa = m.y, j = meta_jidx(m.z);
          float vp[6], ap[6];
          if (pa < 0) {
            vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
            ap[0] = ap[1] = ap[2] = 0.0f;
            ap[3] = r.abase[0];
            ap[4] = r.abase[1];
            ap[5] = r.abase[2];
          } else {
            load6(v + 6 * pa, vp);
            load6(a + 6 * pa, ap);
          }
          const float4 a4 = ct.ax[k];
          const float ax[3] = {a4.x, a4.y, a4.z};
          const float mm = ct.mm[k].x;
          const float vq = j >= 0 ? mm * qd[j] : 0.0f;
          const float aq = j >= 0 ? mm * qdd[j] : 0.0f;
          float vk[6], ak[6];
          rnea_va(Rl + 12 * k, Rl + 12 * k + 9, vp, ap, meta_jtype(m.z), ax, vq, aq, vk, ak);
          store6(v + 6 * k, vk);
          store6(a + 6 * k, ak);
        }
        __syncwarp();
      }
      // pass 2: f = I a + v x* I v
      for (int i = lig; i < n; i += G) {
        const int k = ct.lvm[i].x;
        float I[10], vk[6], ak[6], f[6];
        load_inertia(r, k, I);
        load6(v + 6 * k, vk);
        load6(a + 6 * k, ak);
        rnea_force(I, vk, ak, f);
        store6(F + 6 * k, f);
      }
      __syncwarp();
      // pass 3, tips -> base: F_k = f_k + sum_children X_c^T F_c (a child
      // leaves X^T F in its own v slot, dead after pass 2); S^T F_k goes to
      // the link's a slot (dead too)
      for (int lev = r.nlev - 1; lev >= 0; --lev) {
        const int s1 = ct.lev[lev + 1];
        for (int i = ct.lev[lev] + lig; i < s1; i += G) {
          const int4 m = ct.lvm[i];
          const int k = m.x;
          float f[6];
          load6(F + 6 * k, f);
          const int c1 = m.w >> 16;
          for (int ci = m.w & 0xFFFF; ci < c1; ++ci) {
            const int c = __ldg(r.children + ci);
#pragma unroll
            for (int e = 0; e < 6; ++e) f[e] += v[6 * c + e];
          }
          const float4 a4 = ct.ax[k];
          const float ax[3] = {a4.x, a4.y, a4.z};
          a[6 * k] = St_dot(meta_jtype(m.z), ax, f);
          if (m.y >= 0) {
            float up[6];
            xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, f, up);
            store6(v + 6 * k, up);
          }
        }
        __syncwarp();
      }
      // per joint: tau_j = sum over driven links of m_k S_k^T F_k
      for (int j = lig; j < d; j += G) {
        float t = 0.0f;
        const int e1 = __ldg(r.jl_start + j + 1);
        for (int e = __ldg(r.jl_start + j); e < e1; ++e) {
          const int k = __ldg(r.jl_links + e);
          t = fmaf(ct.mm[k].x, a[6 * k], t);
        }
        qs[j] = t;  // q is dead after FK: stage tau in its slot
      }
    }
    __syncthreads();
    if (A.tau) unstage_rows(base, pl.stride, qoff, A.tau, d, B, b0, cpb);
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
__device__ __forceinline__ void motion_S6(int jt, const float* ax, float* S) {
  S[0] = S[1] = S[2] = S[3] = S[4] = S[5] = 0.0f;
  if (jt == 1) {
    S[0] = ax[0]; S[1] = ax[1]; S[2] = ax[2];
  } else if (jt == 2) {
    S[3] = ax[0]; S[4] = ax[1]; S[5] = ax[2];
  }
}

__device__ __forceinline__ float dot6f(const float* a, const float* b) {
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) s = fmaf(a[i], b[i], s);
  return s;
}

// add the link-frame wrench of a world-frame point gradient g acting at the
// sphere with local centre (sp.xyz) on a link with world rotation R
__device__ __forceinline__ void add_point_wrench(const float* R, float4 sp, const float* g,
                                                 float* w) {
  float f[3], nn[3];
  rotT(R, g, f);
  const float c[3] = {sp.x, sp.y, sp.z};
  cross3(c, f, nn);
  w[0] += nn[0];
  w[1] += nn[1];
  w[2] += nn[2];
  w[3] += f[0];
  w[4] += f[1];
  w[5] += f[2];
}

template <int G>
__global__ void __launch_bounds__(256, 3) fused_bwd_kernel(DevRobot r, BwdArgs A, int cpb) {
  extern __shared__ __align__(128) float smem[];
  const Cta ct = load_cta(r, smem);
  const BwdPlan pl(r.n, r.d);
  float* base = smem + CtaPlan(r.n, r.nlev, r.Sg).total;
  const int lane = threadIdx.x & 31;
  const int lig = lane & (G - 1);
  const int cfg = threadIdx.x / G;
  const int64_t B = A.B;
  const int64_t ntiles = (B + cpb - 1) / cpb;
  float* cs = base + (size_t)cfg * pl.stride;
  const int n = r.n, d = r.d;

  auto stage = [&](int64_t t, int off) {
    const int64_t s0 = t * cpb;
    stage_rows(base, pl.stride, off, A.q, d, B, s0, cpb);
    stage_rows(base, pl.stride, off + d, A.qd, d, B, s0, cpb);
    stage_rows(base, pl.stride, off + 2 * d, A.qdd, d, B, s0, cpb);
    stage_rows(base, pl.stride, off + 3 * d, A.g_tau, d, B, s0, cpb);
    cp_async_commit();
  };
  if ((int64_t)blockIdx.x < ntiles) stage(blockIdx.x, pl.q);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t b0 = tile * cpb;
    const int qoff = (it & 1) ? pl.q2 : pl.q;
    cp_async_wait_all();
    __syncthreads();
    if (tile + gridDim.x < ntiles) stage(tile + gridDim.x, (it & 1) ? pl.q : pl.q2);
    const int64_t b = b0 + cfg;
    const bool live = b < B;
    float* qs = cs + qoff;
    const float* qd = qs + d;
    const float* qdd = qs + 2 * d;
    const float* gt = qs + 3 * d;
    float* Rl = cs + pl.Rl;
    float* Rw = cs + pl.Rw;
    float* v = cs + pl.va;
    float* a = cs + pl.va + 6 * n;
    float* F = cs + pl.F;
    float* Wr = cs + pl.W;
    // ---- local transforms (Rl, copied into Rw) ----
    for (int i = lig; i < n; i += G) {
      const int4 m = ct.lvm[i];
      const int k = m.x, j = meta_jidx(m.z);
      const float2 mm = ct.mm[k];
      const float th = j >= 0 ? fmaf(mm.x, qs[j], mm.y) : 0.0f;
      float T[12];
      local_tf(r, k, meta_jtype(m.z), meta_rotid(m.z), ct.ax[k], th, T);
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        Rl[12 * k + e] = T[e];
        Rw[12 * k + e] = T[e];
      }
    }
    __syncwarp();
    // ---- base -> tips: world poses and the dynamics forward sweep (v, a) ----
    for (int lev = 0; lev < r.nlev; ++lev) {
      const int s1 = ct.lev[lev + 1];
      for (int i = ct.lev[lev] + lig; i < s1; i += G) {
        const int4 m = ct.lvm[i];
        const int k = m.x, pa = m.y, j = meta_jidx(m.z);
        float vp[6], ap[6];
        if (pa < 0) {
          vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
          ap[0] = ap[1] = ap[2] = 0.0f;
          ap[3] = r.abase[0];
          ap[4] = r.abase[1];
          ap[5] = r.abase[2];
        } else {
          float P[12];
          load12(Rw + 12 * pa, P);
          compose_inplace(P, Rw + 12 * k);
          load6(v + 6 * pa, vp);
          load6(a + 6 * pa, ap);
        }
        const float4 a4 = ct.ax[k];
        const float ax[3] = {a4.x, a4.y, a4.z};
        const float mm = ct.mm[k].x;
        const float vq = j >= 0 ? mm * qd[j] : 0.0f;
        const float aq = j >= 0 ? mm * qdd[j] : 0.0f;
        float vk[6], ak[6];
        rnea_va(Rl + 12 * k, Rl + 12 * k + 9, vp, ap, meta_jtype(m.z), ax, vq, aq, vk, ak);
        store6(v + 6 * k, vk);
        store6(a + 6 * k, ak);
      }
      __syncwarp();
    }
    // ---- per link: gradient wrench of the kinematic outputs; force f_k ----
    for (int i = lig; i < n; i += G) {
      const int k = ct.lvm[i].x;
      float w[6] = {0, 0, 0, 0, 0, 0};
      float R[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) R[e] = Rw[12 * k + e];
      if (live && A.g_pose) {
        const float4* g4 = reinterpret_cast<const float4*>(A.g_pose + (b * n + k) * 12);
        const float4 x0 = __ldg(g4), x1 = __ldg(g4 + 1), x2 = __ldg(g4 + 2);
        const float gg[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y,
                              x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
        float Gm[9];  // R^T Rbar
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int jj = 0; jj < 3; ++jj)
            Gm[3 * ii + jj] =
                fmaf(R[6 + ii], gg[6 + jj], fmaf(R[3 + ii], gg[3 + jj], R[ii] * gg[jj]));
        w[0] = Gm[7] - Gm[5];
        w[1] = Gm[2] - Gm[6];
        w[2] = Gm[3] - Gm[1];
        rotT(R, gg + 9, w + 3);
      }
      if (live && A.g_sph) {
        const int e1 = __ldg(r.ls_start + k + 1);
        for (int e = __ldg(r.ls_start + k); e < e1; ++e) {
          const int s = __ldg(r.ls_sph + e);
          const float* g = A.g_sph + (b * r.S + s) * 3;
          const float gg[3] = {__ldg(g), __ldg(g + 1), __ldg(g + 2)};
          add_point_wrench(R, __ldg(r.sph + s), gg, w);
        }
      }
      store6(Wr + 6 * k, w);
      float I[10], vk[6], ak[6], f[6];
      load_inertia(r, k, I);
      load6(v + 6 * k, vk);
      load6(a + 6 * k, ak);
      rnea_force(I, vk, ak, f);
      store6(F + 6 * k, f);
    }
    __syncwarp();
    if (live && A.g_dmin && lig == 0) {
      const int wp = A.worst[b];
      const float gd = A.g_dmin[b];
      if (wp >= 0 && wp < r.P) {
        const int2 ij = __ldg(r.pairs + wp);
        const float4 si = __ldg(r.sph + ij.x), sj = __ldg(r.sph + ij.y);
        const int l1 = __ldg(r.sph_link + ij.x), l2 = __ldg(r.sph_link + ij.y);
        float ci[3], cj[3];
        const float li[3] = {si.x, si.y, si.z}, lj[3] = {sj.x, sj.y, sj.z};
        rot(Rw + 12 * l1, li, ci);
        rot(Rw + 12 * l2, lj, cj);
        const float dx = (ci[0] + Rw[12 * l1 + 9]) - (cj[0] + Rw[12 * l2 + 9]);
        const float dy = (ci[1] + Rw[12 * l1 + 10]) - (cj[1] + Rw[12 * l2 + 10]);
        const float dz = (ci[2] + Rw[12 * l1 + 11]) - (cj[2] + Rw[12 * l2 + 11]);
        const float nrm = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
        const float sc = nrm > 0.0f ? gd / nrm : 0.0f;
        const float u[3] = {dx * sc, dy * sc, dz * sc};
        const float mu[3] = {-u[0], -u[1], -u[2]};
        add_point_wrench(Rw + 12 * l1, si, u, Wr + 6 * l1);
        add_point_wrench(Rw + 12 * l2, sj, mu, Wr + 6 * l2);
      }
    }
    __syncwarp();
    // ---- tips -> base: accumulated force F (children leave X^T F in `up`) ----
    float* up = cs + pl.up;  // Rw is dead from here on
    for (int lev = r.nlev - 1; lev >= 0; --lev) {
      const int s1 = ct.lev[lev + 1];
      for (int i = ct.lev[lev] + lig; i < s1; i += G) {
        const int4 m = ct.lvm[i];
        const int k = m.x;
        float f[6];
        load6(F + 6 * k, f);
        const int c1 = m.w >> 16;
        for (int ci = m.w & 0xFFFF; ci < c1; ++ci) {
          const int c = __ldg(r.children + ci);
#pragma unroll
          for (int e = 0; e < 6; ++e) f[e] += up[6 * c + e];
        }
        store6(F + 6 * k, f);
        if (m.y >= 0) {
          float u6[6];
          xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, f, u6);
          store6(up + 6 * k, u6);
        }
      }
      __syncwarp();
    }
    float* vb = cs + pl.vb;
    float* lq = cs + pl.lq;
    // ---- adjoint of the force sweep, base -> tips (F slot: F -> Fbar) ----
    for (int lev = 0; lev < r.nlev; ++lev) {
      const int s1 = ct.lev[lev + 1];
      for (int i = ct.lev[lev] + lig; i < s1; i += G) {
        const int4 m = ct.lvm[i];
        const int k = m.x, pa = m.y, j = meta_jidx(m.z);
        const float4 a4 = ct.ax[k];
        const float ax[3] = {a4.x, a4.y, a4.z};
        float S[6];
        motion_S6(meta_jtype(m.z), ax, S);
        const float tb = j >= 0 ? ct.mm[k].x * gt[j] : 0.0f;
        float XF[6], cS[6], Fk[6];
        if (pa >= 0) {
          float Fp[6];
          load6(F + 6 * pa, Fp);
          xf_motion(Rl + 12 * k, Rl + 12 * k + 9, Fp, XF);
        } else {
          XF[0] = XF[1] = XF[2] = XF[3] = XF[4] = XF[5] = 0.0f;
        }
        load6(F + 6 * k, Fk);
        crf(S, Fk, cS);
        lq[3 * k] = dot6f(XF, cS);
#pragma unroll
        for (int e = 0; e < 6; ++e) F[6 * k + e] = fmaf(S[e], tb, XF[e]);
      }
      __syncwarp();
    }
    // ---- adjoint of the per-link force (F slot: Fbar -> abar; vbar) ----
    for (int i = lig; i < n; i += G) {
      const int k = ct.lvm[i].x;
      float I[10], Fb[6], vk[6], Iv[6], t1[6], t2[6], t3[6], ab[6];
      load_inertia(r, k, I);
      load6(F + 6 * k, Fb);
      load6(v + 6 * k, vk);
      inertia_mul(I, Fb, ab);
      inertia_mul(I, vk, Iv);
      crf(Fb, Iv, t1);
      crm(vk, Fb, t2);
      inertia_mul(I, t2, t3);
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        F[6 * k + e] = ab[e];
        vb[6 * k + e] = -t1[e] - t3[e];
      }
    }
    __syncwarp();
    // ---- adjoint of the velocity/acceleration sweep and of FK, tips -> base ----
    for (int lev = r.nlev - 1; lev >= 0; --lev) {
      const int s1 = ct.lev[lev + 1];
      for (int i = ct.lev[lev] + lig; i < s1; i += G) {
        const int4 m = ct.lvm[i];
        const int k = m.x, pa = m.y, j = meta_jidx(m.z);
        const float4 a4 = ct.ax[k];
        const float ax[3] = {a4.x, a4.y, a4.z};
        float S[6];
        motion_S6(meta_jtype(m.z), ax, S);
        const float vq = j >= 0 ? ct.mm[k].x * qd[j] : 0.0f;
        float ab[6], vbk[6], w[6];
        load6(F + 6 * k, ab);
        load6(vb + 6 * k, vbk);
        load6(Wr + 6 * k, w);
        const int c1 = m.w >> 16;
        for (int ci = m.w & 0xFFFF; ci < c1; ++ci) {
          const int c = __ldg(r.children + ci);
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            ab[e] += F[6 * c + e];
            vbk[e] += vb[6 * c + e];
            w[e] += Wr[6 * c + e];
          }
        }
        float t[6], vk[6];
        crf(S, ab, t);
#pragma unroll
        for (int e = 0; e < 6; ++e) vbk[e] = fmaf(vq, t[e], vbk[e]);
        const float gqdd = dot6f(S, ab);
        load6(v + 6 * k, vk);
        crf(vk, ab, t);
        const float gqd = dot6f(S, vbk) - dot6f(S, t);
        float vp[6], ap[6];
        if (pa < 0) {
          vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
          ap[0] = ap[1] = ap[2] = 0.0f;
          ap[3] = r.abase[0];
          ap[4] = r.abase[1];
          ap[5] = r.abase[2];
        } else {
          load6(v + 6 * pa, vp);
          load6(a + 6 * pa, ap);
        }
        float Xa[6], Xv[6], c6[6];
        xf_motion(Rl + 12 * k, Rl + 12 * k + 9, ap, Xa);
        xf_motion(Rl + 12 * k, Rl + 12 * k + 9, vp, Xv);
        float gq = lq[3 * k];
        crm(S, Xa, c6);
        gq -= dot6f(ab, c6);
        crm(S, Xv, c6);
        gq -= dot6f(vbk, c6);
        gq += dot6f(S, w);
        lq[3 * k] = gq;
        lq[3 * k + 1] = gqd;
        lq[3 * k + 2] = gqdd;
        if (pa >= 0) {
          float u6[6];
          xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, ab, u6);
          store6(F + 6 * k, u6);
          xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, vbk, u6);
          store6(vb + 6 * k, u6);
          xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, w, u6);
          store6(Wr + 6 * k, u6);
        }
      }
      __syncwarp();
    }
    // ---- per joint (mimic joints sum their links); stage in q slots ----
    for (int jj = lig; jj < d; jj += G) {
      float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
      const int e1 = __ldg(r.jl_start + jj + 1);
      for (int e = __ldg(r.jl_start + jj); e < e1; ++e) {
        const int k = __ldg(r.jl_links + e);
        const float mm = ct.mm[k].x;
        g0 = fmaf(mm, lq[3 * k], g0);
        g1 = fmaf(mm, lq[3 * k + 1], g1);
        g2 = fmaf(mm, lq[3 * k + 2], g2);
      }
      qs[jj] = g0;
      qs[d + jj] = g1;
      qs[2 * d + jj] = g2;
    }
    __syncthreads();
    unstage_rows(base, pl.stride, qoff, A.gq, d, B, b0, cpb);
    unstage_rows(base, pl.stride, qoff + d, A.gqd, d, B, b0, cpb);
    unstage_rows(base, pl.stride, qoff + 2 * d, A.gqdd, d, B, b0, cpb);
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int G>
static cudaError_t fwd_launch_t(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                                const FusedShape& sh, cudaStream_t s) {
  auto kern = fused_fwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sh.smem);
  if (e != cudaSuccess) return e;
  kern<<<sh.grid, sh.cpb * G, sh.smem, s>>>(r, ps, a, sh.cpb);
  return cudaGetLastError();
}

template <int G>
static cudaError_t bwd_launch_t(const DevRobot& r, const BwdArgs& a, const FusedShape& sh,
                                cudaStream_t s) {
  auto kern = fused_bwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sh.smem);
  if (e != cudaSuccess) return e;
  kern<<<sh.grid, sh.cpb * G, sh.smem, s>>>(r, a, sh.cpb);
  return cudaGetLastError();
}

cudaError_t launch_fused_fwd(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                             const FusedShape& sh, cudaStream_t s) {
  switch (sh.G) {
    case 4: return fwd_launch_t<4>(r, ps, a, sh, s);
    case 8: return fwd_launch_t<8>(r, ps, a, sh, s);
    case 16: return fwd_launch_t<16>(r, ps, a, sh, s);
    case 32: return fwd_launch_t<32>(r, ps, a, sh, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fused_bwd(const DevRobot& r, const BwdArgs& a, const FusedShape& sh,
                             cudaStream_t s) {
  switch (sh.G) {
    case 4: return bwd_launch_t<4>(r, a, sh, s);
    case 8: return bwd_launch_t<8>(r, a, sh, s);
    case 16: return bwd_launch_t<16>(r, a, sh, s);
    case 32: return bwd_launch_t<32>(r, a, sh, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int G>
static cudaError_t occ_fwd_t(int cpb, size_t smem, int* out) {
  auto kern = fused_fwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, cpb * G, smem);
}
template <int G>
static cudaError_t occ_bwd_t(int cpb, size_t smem, int* out) {
  auto kern = fused_bwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, cpb * G, smem);
}

cudaError_t fused_fwd_max_blocks_per_sm(int G, int cpb, size_t smem, int* out) {
  switch (G) {
    case 4: return occ_fwd_t<4>(cpb, smem, out);
    case 8: return occ_fwd_t<8>(cpb, smem, out);
    case 16: return occ_fwd_t<16>(cpb, smem, out);
    case 32: return occ_fwd_t<32>(cpb, smem, out);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t fused_bwd_max_blocks_per_sm(int G, int cpb, size_t smem, int* out) {
  switch (G) {
    case 4: return occ_bwd_t<4>(cpb, smem, out);
    case 8: return occ_bwd_t<8>(cpb, smem, out);
    case 16: return occ_bwd_t<16>(cpb, smem, out);
    case 32: return occ_bwd_t<32>(cpb, smem, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wbe
