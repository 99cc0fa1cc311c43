// wbe_api.cu -- host side of libwbe.so: the C ABI declared in include/wbe.h.
//
// wb_load_robot validates the descriptor and builds, once per robot:
//   * the topology cache of Sec. 6.1.2: tree levels (links of equal depth),
//     children lists, the links driven by each joint (mimic joints, Alg. 1
//     "jointMap"), the spheres of each link;
//   * compact float parameters: fixed transforms (R, p), unit axes, the
//     10-float spatial inertia (m, m c, inertia about the link origin) with
//     payload point masses added (spatial inertias are additive);
//   * the row-major sorted pair list, its 4x4 sphere-group blocks and a
//     per-lane block schedule for each fused launch width;
// and copies them to the device in one allocation.
#include "../../include/wbe.h"
#include "wbe_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace wbe;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(WB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Runs with the robot's device current and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------------------
// the robot handle
// ---------------------------------------------------------------------------
struct wb_robot {
  int device = 0;
  int num_sms = 0;
  DevRobot dev{};
  void* dmem = nullptr;
  size_t dbytes = 0;
  float* d_inert = nullptr;   // device inertia array (inside dmem)
  PairSchedule sched[4]{};    // G = 4, 8, 16, 32
  PairSchedule32 sched32{};   // the pair kernel's (byte-offset encoding)
  wb_robot_info info{};
  // host copies needed by set_inertials
  int n = 0, S = 0;
  float* h_stage = nullptr;   // pinned staging buffer for inertia uploads
  cudaEvent_t stage_evt = nullptr;
  bool stage_pending = false;
  // without / with pair bits, set on first use (any host thread may be first)
  std::atomic<int> pair_warps_default[2] = {0, 0};
};

static int sched_slot(int G) { return G == 4 ? 0 : G == 8 ? 1 : G == 16 ? 2 : G == 32 ? 3 : -1; }

// Sub-allocator for the single device block.
struct Packer {
  std::vector<char> host;
  struct Item {
    size_t off;
    const void** slot;
  };
  std::vector<Item> items;
  size_t add(const void* src, size_t bytes, const void** slot) {
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + std::max<size_t>(bytes, 16));
    if (bytes) std::memcpy(host.data() + off, src, bytes);
    items.push_back({off, slot});
    return off;
  }
  template <class T>
  size_t add_vec(const std::vector<T>& v, const T** slot) {
    return add(v.data(), v.size() * sizeof(T), reinterpret_cast<const void**>(slot));
  }
};

// 10-float compact spatial inertia at the link origin, point masses added
static int compact_inertia(const wb_inertial* in, int n, std::vector<float>& out) {
  if (!in || !in->mass || !in->com || !in->inertia)
    return fail(WB_EINVAL, "inertial: mass, com and inertia are required");
  std::vector<double> acc(10 * (size_t)n, 0.0);
  auto add_body = [&](int k, double m, const double* c, const double* Ic) {
    double* o = &acc[10 * (size_t)k];
    const double cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    o[0] += m;
    o[1] += m * c[0];
    o[2] += m * c[1];
    o[3] += m * c[2];
    // Io = Ic + m (|c|^2 I - c c^T)
    o[4] += (Ic ? Ic[0] : 0.0) + m * (cc - c[0] * c[0]);
    o[5] += (Ic ? Ic[1] : 0.0) + m * (cc - c[1] * c[1]);
    o[6] += (Ic ? Ic[2] : 0.0) + m * (cc - c[2] * c[2]);
    o[7] += (Ic ? Ic[3] : 0.0) - m * c[0] * c[1];
    o[8] += (Ic ? Ic[4] : 0.0) - m * c[0] * c[2];
    o[9] += (Ic ? Ic[5] : 0.0) - m * c[1] * c[2];
  };
  for (int k = 0; k < n; ++k) {
    const double m = in->mass[k];
    if (!std::isfinite(m) || m < 0) return fail(WB_EINVAL, "inertial: bad mass at link %d", k);
    for (int i = 0; i < 3; ++i)
      if (!std::isfinite(in->com[3 * k + i])) return fail(WB_EINVAL, "inertial: bad com %d", k);
    for (int i = 0; i < 6; ++i)
      if (!std::isfinite(in->inertia[6 * k + i]))
        return fail(WB_EINVAL, "inertial: bad inertia at link %d", k);
    add_body(k, m, in->com + 3 * k, in->inertia + 6 * k);
  }
  if (in->n_points < 0) return fail(WB_EINVAL, "inertial: n_points < 0");
  if (in->n_points > 0 && (!in->point_link || !in->point_mass || !in->point_pos))
    return fail(WB_EINVAL, "inertial: point mass arrays are required when n_points > 0");
  for (int m = 0; m < in->n_points; ++m) {
    const int l = in->point_link[m];
    if (l < 0 || l >= n) return fail(WB_ERANGE, "inertial: point mass %d on link %d", m, l);
    if (!std::isfinite(in->point_mass[m]) || in->point_mass[m] < 0)
      return fail(WB_EINVAL, "inertial: bad point mass %d", m);
    add_body(l, in->point_mass[m], in->point_pos + 3 * m, nullptr);
  }
  out.resize(acc.size());
  for (size_t i = 0; i < acc.size(); ++i) out[i] = (float)acc[i];
  return WB_OK;
}

// Deal the pair blocks of one launch width G to the lanes.  Blocks of column
// class gj mod C (C = min(G, 8)) go to the lanes l with l mod C == class, so
// that the 8 lanes of a shared-memory phase read distinct bank groups; each
// class is sorted by row group gi (a lane reloads its row spheres only when
// gi changes) and cut into equal contiguous runs.
static void build_schedule(int G, const std::vector<uint32_t>& bx, std::vector<uint2>& ent,
                           int& rounds) {
  const int C = std::min(G, 8);
  const int per = G / C;
  std::vector<std::vector<int>> lanes(G);
  for (int c = 0; c < C; ++c) {
    std::vector<int> cls;
    for (int b = 0; b < (int)bx.size(); ++b)
      if ((int)((bx[b] >> 8) & 0xFF) % C == c) cls.push_back(b);
    // row group gi first, then column group gj
    auto key = [&](int b) { return ((bx[b] & 0xFF) << 8) | ((bx[b] >> 8) & 0xFF); };
    std::stable_sort(cls.begin(), cls.end(), [&](int a, int b) { return key(a) < key(b); });
    const size_t m = cls.size();
    for (int t = 0; t < per; ++t) {
      const size_t lo = m * t / per, hi = m * (t + 1) / per;
      for (size_t i = lo; i < hi; ++i) lanes[c + t * C].push_back(cls[i]);
    }
  }
  // even out lanes whose class is larger than average: move the tail of the
  // longest lane to the shortest until the spread is at most one block
  for (int it = 0; it < 100000; ++it) {
    int lo = 0, hi = 0;
    for (int l = 1; l < G; ++l) {
      if (lanes[l].size() < lanes[lo].size()) lo = l;
      if (lanes[l].size() > lanes[hi].size()) hi = l;
    }
    if (lanes[hi].size() <= lanes[lo].size() + 1) break;
    lanes[lo].push_back(lanes[hi].back());
    lanes[hi].pop_back();
  }
  rounds = 0;
  for (int l = 0; l < G; ++l) rounds = std::max(rounds, (int)lanes[l].size());
  // one extra all-null round: kernels may prefetch round r + 1 unguarded
  ent.assign((size_t)(rounds + 1) * G, uint2{0u, 0u});
  for (int l = 0; l < G; ++l)
    for (size_t i = 0; i < lanes[l].size(); ++i) {
      const int b = lanes[l][i];
      ent[i * G + l] = uint2{bx[b], (uint32_t)b};
    }
}

extern "C" {

int wb_version(void) { return 102; }

const char* wb_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// Everything wb_load_robot computes on the host, before touching a device.
struct HostPlan {
  int n = 0, d = 0, S = 0, P = 0, nlev = 0, maxw = 0, Sg = 0;
  float g[3];
  double reach = 0.0;
  std::vector<int16_t> parent, jidx, lev_start, lev_links, child_start, children, jl_start,
      jl_links, ls_start, ls_sph, sph_link;
  std::vector<int8_t> jtype, rot_id;
  std::vector<float> axis, Tf, mimic, inert;
  std::vector<float4> sp, grp_rad, grp_loc;
  std::vector<int16_t> grp_link;
  std::vector<int2> pairs_dev;
  std::vector<uint32_t> bx;
  std::vector<int32_t> blk_pidx;
  std::vector<int4> lvm;
  std::vector<int2> dfs, dfs_kj;
  std::vector<int> lmeta, chain_m;
  std::vector<int16_t> chain_start, chain;
  int maxdepth = 0;
  int mimic_shared = 0;
  double r_max = 0.0;
  // segmented-sweep plans (G = 2, 4, 8)
  std::vector<int16_t> dfs_pos, dfs_end, seg_slot, seg_slot_link;
  int seg_ok = 0;
  int seg_ns[3] = {0, 0, 0};
  int16_t seg_pos[3][9] = {};
};

// Cut the DFS order into G contiguous segments minimising the largest
// segment cost = owned links + 0.7 x replayed ancestors (the depth of the
// segment's first link): a replayed link does the pre-order without the
// link's own force / adjoint terms, then a full post-order.  Links held by
// more than one segment (the proper ancestors of a segment's first link)
// that drive a joint get an output slot.
static void plan_segments(HostPlan& H, int t) {
  const int n = H.n, G = 2 << t;
  if (H.mimic_shared || n < G) return;
  const double kInf = 1e300;
  auto cost = [&](int s, int e) { return (e - s) + 0.7 * H.dfs[s].y; };
  std::vector<double> best((size_t)(G + 1) * (n + 1), kInf);
  std::vector<int> arg((size_t)(G + 1) * (n + 1), 0);
  auto at = [&](int g, int e) { return (size_t)g * (n + 1) + e; };
  best[at(0, 0)] = 0.0;
  for (int g = 1; g <= G; ++g)
    for (int e = g; e <= n; ++e)
      for (int s0 = g - 1; s0 < e; ++s0) {
        const double v = std::max(best[at(g - 1, s0)], cost(s0, e));
        if (v < best[at(g, e)]) {
          best[at(g, e)] = v;
          arg[at(g, e)] = s0;
        }
      }
  int e = n;
  H.seg_pos[t][G] = (int16_t)n;
  for (int g = G; g >= 1; --g) {
    e = arg[at(g, e)];
    H.seg_pos[t][g - 1] = (int16_t)e;
  }
  int16_t* slot = &H.seg_slot[(size_t)t * n];
  int16_t* link = &H.seg_slot_link[(size_t)t * n];
  int ns = 0;
  for (int g = 1; g < G; ++g) {
    const int k0 = H.dfs[H.seg_pos[t][g]].x;
    for (int c = H.chain_start[k0]; c < H.chain_start[k0 + 1] - 1; ++c) {
      const int a = H.chain[c];
      if (H.jidx[a] >= 0 && slot[a] < 0) {
        slot[a] = (int16_t)ns;
        link[ns++] = (int16_t)a;
      }
    }
  }
  H.seg_ns[t] = ns;
  H.seg_ok |= 1 << t;
}

static int plan_robot(const wb_tree* tree, const wb_spheres* sph, const wb_pairs* pairs,
                      const wb_inertial* inertial, HostPlan& H) {
  if (!tree || !sph || !pairs || !inertial) return fail(WB_EINVAL, "NULL descriptor");
  const int n = tree->n_links;
  if (n <= 0) return fail(WB_EINVAL, "n_links must be positive");
  if (n > WB_MAX_LINKS) return fail(WB_ETOOBIG, "n_links %d > %d", n, WB_MAX_LINKS);
  if (!tree->parent || !tree->joint_type || !tree->axis || !tree->T_fixed || !tree->joint_index)
    return fail(WB_EINVAL, "tree: parent, joint_type, axis, T_fixed, joint_index are required");

  // ---- tree ----
  std::vector<int16_t> parent(n), jidx(n);
  std::vector<int8_t> jtype(n), rot_id(n);
  std::vector<float> axis(4 * (size_t)n, 0.0f), Tf(12 * (size_t)n), mimic(2 * (size_t)n);
  int d = 0;
  for (int k = 0; k < n; ++k) {
    const int pa = tree->parent[k];
    if (pa < -1 || pa >= k) return fail(WB_ETOPO, "parent[%d] = %d must be in [-1, %d)", k, pa, k);
    parent[k] = (int16_t)pa;
    const int jt = tree->joint_type[k];
    if (jt < 0 || jt > 2) return fail(WB_ETOPO, "joint_type[%d] = %d", k, jt);
    jtype[k] = (int8_t)jt;
    const int j = tree->joint_index[k];
    if (jt == 0 && j != -1) return fail(WB_ETOPO, "fixed link %d has joint_index %d", k, j);
    if (jt != 0 && (j < 0 || j >= n))
      return fail(WB_ETOPO, "joint_index[%d] = %d out of range", k, j);
    jidx[k] = (int16_t)j;
    d = std::max(d, j + 1);
    const double* ax = tree->axis + 3 * k;
    if (jt != 0) {
      const double nrm = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
      if (!std::isfinite(nrm) || std::fabs(nrm - 1.0) > 1e-5)
        return fail(WB_EINVAL, "axis of link %d is not unit (|a| = %g)", k, nrm);
      for (int i = 0; i < 3; ++i) axis[4 * k + i] = (float)(ax[i] / nrm);
    }
    const double* T = tree->T_fixed + 12 * k;
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(T[i])) return fail(WB_EINVAL, "T_fixed of link %d not finite", k);
    double dev = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int jj = 0; jj < 3; ++jj) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += T[3 * m + i] * T[3 * m + jj];
        dev = std::max(dev, std::fabs(s - (i == jj ? 1.0 : 0.0)));
      }
    if (dev > 1e-5) return fail(WB_EINVAL, "T_fixed rotation of link %d not orthonormal", k);
    bool ident = true;
    for (int i = 0; i < 9; ++i) {
      Tf[12 * k + i] = (float)T[i];
      if (T[i] != ((i % 4 == 0) ? 1.0 : 0.0)) ident = false;
    }
    for (int i = 9; i < 12; ++i) Tf[12 * k + i] = (float)T[i];
    rot_id[k] = ident ? 1 : 0;
    mimic[2 * k] = tree->mimic_mult ? (float)tree->mimic_mult[k] : 1.0f;
    mimic[2 * k + 1] = tree->mimic_offset ? (float)tree->mimic_offset[k] : 0.0f;
    if (!std::isfinite(mimic[2 * k]) || !std::isfinite(mimic[2 * k + 1]))
      return fail(WB_EINVAL, "mimic parameters of link %d not finite", k);
  }
  // every joint must drive at least one link
  std::vector<std::vector<int16_t>> jl(d);
  for (int k = 0; k < n; ++k)
    if (jidx[k] >= 0) jl[jidx[k]].push_back((int16_t)k);
  for (int j = 0; j < d; ++j)
    if (jl[j].empty()) return fail(WB_ETOPO, "joint %d drives no link", j);
  float g[3] = {0.0f, 0.0f, -9.81f};
  if (tree->gravity)
    for (int i = 0; i < 3; ++i) g[i] = (float)tree->gravity[i];

  // levels, children
  std::vector<int> depth(n);
  int nlev = 0;
  for (int k = 0; k < n; ++k) {
    depth[k] = parent[k] < 0 ? 0 : depth[parent[k]] + 1;
    nlev = std::max(nlev, depth[k] + 1);
  }
  std::vector<int16_t> lev_start(nlev + 1, 0), lev_links;
  int maxw = 0;
  for (int l = 0; l < nlev; ++l) {
    lev_start[l] = (int16_t)lev_links.size();
    for (int k = 0; k < n; ++k)
      if (depth[k] == l) lev_links.push_back((int16_t)k);
    maxw = std::max(maxw, (int)lev_links.size() - lev_start[l]);
  }
  lev_start[nlev] = (int16_t)lev_links.size();
  std::vector<int16_t> child_start(n + 1, 0), children;
  for (int k = 0; k < n; ++k) {
    child_start[k] = (int16_t)children.size();
    for (int c = k + 1; c < n; ++c)
      if (parent[c] == k) children.push_back((int16_t)c);
  }
  child_start[n] = (int16_t)children.size();
  std::vector<int16_t> jl_start(d + 1, 0), jl_links;
  for (int j = 0; j < d; ++j) {
    jl_start[j] = (int16_t)jl_links.size();
    jl_links.insert(jl_links.end(), jl[j].begin(), jl[j].end());
  }
  jl_start[d] = (int16_t)jl_links.size();

  // ---- spheres ----
  const int S = sph->n_spheres;
  if (S < 0) return fail(WB_EINVAL, "n_spheres < 0");
  if (S > WB_MAX_SPHERES) return fail(WB_ETOOBIG, "n_spheres %d > %d", S, WB_MAX_SPHERES);
  if (S > 0 && (!sph->link || !sph->center || !sph->radius))
    return fail(WB_EINVAL, "spheres: link, center, radius are required");
  std::vector<float4> sp(std::max(S, 1));
  std::vector<int16_t> sph_link(std::max(S, 1), 0);
  double max_c = 0.0, max_r = 0.0;
  for (int s = 0; s < S; ++s) {
    const int l = sph->link[s];
    if (l < 0 || l >= n) return fail(WB_ERANGE, "sphere %d on link %d", s, l);
    const double* c = sph->center + 3 * s;
    const double rr = sph->radius[s];
    if (!std::isfinite(c[0]) || !std::isfinite(c[1]) || !std::isfinite(c[2]) ||
        !std::isfinite(rr) || rr < 0)
      return fail(WB_EINVAL, "sphere %d: bad centre or radius", s);
    sp[s] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)rr);
    sph_link[s] = (int16_t)l;
    max_c = std::max(max_c, std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]));
    max_r = std::max(max_r, rr);
  }
  std::vector<int16_t> ls_start(n + 1, 0), ls_sph;
  for (int k = 0; k < n; ++k) {
    ls_start[k] = (int16_t)ls_sph.size();
    for (int s = 0; s < S; ++s)
      if (sph_link[s] == k) ls_sph.push_back((int16_t)s);
  }
  ls_start[n] = (int16_t)ls_sph.size();
  if (ls_sph.empty()) ls_sph.push_back(0);

  // ---- pairs: sort row-major, validate ----
  std::vector<std::pair<int, int>> pl;
  if (pairs->mask && pairs->pairs) return fail(WB_EINVAL, "pairs: give a list or a mask, not both");
  if (pairs->mask) {
    for (int i = 0; i < S; ++i)
      for (int j = i + 1; j < S; ++j)
        if (pairs->mask[(size_t)i * S + j]) pl.emplace_back(i, j);
  } else {
    if (pairs->n_pairs < 0) return fail(WB_EINVAL, "n_pairs < 0");
    if (pairs->n_pairs > 0 && !pairs->pairs) return fail(WB_EINVAL, "pairs: list is NULL");
    for (int p = 0; p < pairs->n_pairs; ++p) {
      const int i = pairs->pairs[2 * p], j = pairs->pairs[2 * p + 1];
      if (i < 0 || j < 0 || i >= S || j >= S)
        return fail(WB_ERANGE, "pair %d = (%d, %d) out of range (S = %d)", p, i, j, S);
      if (i >= j) return fail(WB_ERANGE, "pair %d = (%d, %d) must have i < j", p, i, j);
      pl.emplace_back(i, j);
    }
    std::sort(pl.begin(), pl.end());
    for (size_t p = 1; p < pl.size(); ++p)
      if (pl[p] == pl[p - 1])
        return fail(WB_ERANGE, "duplicate pair (%d, %d)", pl[p].first, pl[p].second);
  }
  const int P = (int)pl.size();
  std::vector<int2> pairs_dev(std::max(P, 1), int2{0, 0});
  for (int p = 0; p < P; ++p) pairs_dev[p] = int2{pl[p].first, pl[p].second};

  // ---- 4x4 group blocks ----
  const int Sg = std::max((S + 3) / 4, 1);
  std::vector<float4> grp_rad(Sg, make_float4(0, 0, 0, 0));
  for (int s = 0; s < S; ++s) (&grp_rad[s / 4].x)[s % 4] = sp[s].w;
  // A group whose spheres all sit on one link gets a bounding sphere in that
  // link's frame, computed here once (the pair stage then moves it with the
  // link); other groups are bounded per configuration.  Centre: the better
  // of the centroid and a Badoiu-Clarkson minimax iteration; radius: the
  // largest |c_s - C| + r_s from the float centre, rounded up.
  std::vector<float4> grp_loc(Sg, make_float4(0, 0, 0, 0));
  std::vector<int16_t> grp_link(Sg, -1);
  for (int g = 0; g < Sg; ++g) {
    const int s0 = 4 * g, s1 = std::min(S, s0 + 4);
    if (s1 <= s0) continue;
    bool one = true;
    for (int q = s0 + 1; q < s1; ++q) one = one && sph_link[q] == sph_link[s0];
    if (!one) continue;
    auto radius = [&](const double* C) {
      double R = 0.0;
      for (int q = s0; q < s1; ++q) {
        const double dx = sp[q].x - C[0], dy = sp[q].y - C[1], dz = sp[q].z - C[2];
        R = std::max(R, std::sqrt(dx * dx + dy * dy + dz * dz) + (double)sp[q].w);
      }
      return R;
    };
    double cen[3] = {0, 0, 0};
    for (int q = s0; q < s1; ++q) {
      cen[0] += sp[q].x / (s1 - s0);
      cen[1] += sp[q].y / (s1 - s0);
      cen[2] += sp[q].z / (s1 - s0);
    }
    double best[3] = {cen[0], cen[1], cen[2]}, bestR = radius(cen);
    double C[3] = {cen[0], cen[1], cen[2]};
    for (int it = 0; it < 200; ++it) {  // step towards the far point of the farthest sphere
      int far = s0;
      double fd = -1.0;
      for (int q = s0; q < s1; ++q) {
        const double dx = sp[q].x - C[0], dy = sp[q].y - C[1], dz = sp[q].z - C[2];
        const double dq = std::sqrt(dx * dx + dy * dy + dz * dz) + sp[q].w;
        if (dq > fd) {
          fd = dq;
          far = q;
        }
      }
      const double dx = sp[far].x - C[0], dy = sp[far].y - C[1], dz = sp[far].z - C[2];
      const double nn = std::sqrt(dx * dx + dy * dy + dz * dz);
      const double k = nn > 0.0 ? (nn + sp[far].w) / nn : 0.0;
      const double step = 1.0 / (it + 2);
      C[0] += step * dx * k;
      C[1] += step * dy * k;
      C[2] += step * dz * k;
      const double R = radius(C);
      if (R < bestR) {
        bestR = R;
        best[0] = C[0];
        best[1] = C[1];
        best[2] = C[2];
      }
    }
    const float fc[3] = {(float)best[0], (float)best[1], (float)best[2]};
    const double dc[3] = {fc[0], fc[1], fc[2]};
    const float R = std::nextafter((float)radius(dc), INFINITY);
    grp_loc[g] = make_float4(fc[0], fc[1], fc[2], R);
    grp_link[g] = sph_link[s0];
  }
  std::vector<int> blk_of((size_t)Sg * Sg, -1);
  std::vector<uint32_t> bx;  // gi | gj << 8 | mask << 16
  std::vector<int32_t> blk_pidx;
  for (int p = 0; p < P; ++p) {
    const int i = pl[p].first, j = pl[p].second;
    const int gi = i / 4, gj = j / 4;
    int& b = blk_of[(size_t)gi * Sg + gj];
    if (b < 0) {
      b = (int)bx.size();
      bx.push_back((uint32_t)gi | ((uint32_t)gj << 8));
      blk_pidx.insert(blk_pidx.end(), 16, -1);
    }
    const int bit = 4 * (i % 4) + (j % 4);
    bx[b] |= 1u << (16 + bit);
    blk_pidx[16 * (size_t)b + bit] = p;
  }
  if (blk_pidx.empty()) blk_pidx.assign(16, -1);
  if (bx.size() > 65535) return fail(WB_ETOOBIG, "%zu pair blocks > 65535", bx.size());

  // ---- inertia ----
  std::vector<float> inert;
  int rc = compact_inertia(inertial, n, inert);
  if (rc != WB_OK) return rc;

  // pair filter margin: a bound on the float rounding of the squared-distance
  // test, scaled with the robot's reach
  double reach = 0.0;
  {
    std::vector<double> rk(n, 0.0);
    for (int k = 0; k < n; ++k) {
      const double* T = tree->T_fixed + 12 * k;
      const double len = std::sqrt(T[9] * T[9] + T[10] * T[10] + T[11] * T[11]);
      rk[k] = (parent[k] < 0 ? 0.0 : rk[parent[k]]) + len;
      reach = std::max(reach, rk[k]);
    }
    reach += max_c + max_r;
  }

  H.n = n;
  H.d = d;
  H.S = S;
  H.P = P;
  H.nlev = nlev;
  H.maxw = maxw;
  H.Sg = Sg;
  for (int i = 0; i < 3; ++i) H.g[i] = g[i];
  H.reach = reach;
  H.r_max = max_r;
  H.lvm.resize(n);
  for (int i = 0; i < n; ++i) {
    const int k = lev_links[i];
    const int meta = (jidx[k] + 1) | ((int)jtype[k] << 16) | ((int)rot_id[k] << 24);
    H.lvm[i] = make_int4(k, parent[k], meta, child_start[k] | (child_start[k + 1] << 16));
  }
  // depth-first pre-order (children in index order) and ancestor chains
  {
    std::vector<int> stack;
    for (int k = n - 1; k >= 0; --k)
      if (parent[k] < 0) stack.push_back(k);
    while (!stack.empty()) {
      const int k = stack.back();
      stack.pop_back();
      H.dfs.push_back(make_int2(k, depth[k]));
      for (int c = n - 1; c > k; --c)
        if (parent[c] == k) stack.push_back(c);
    }
    H.maxdepth = nlev;
    H.chain_start.assign(n + 1, 0);
    for (int k = 0; k < n; ++k) {
      H.chain_start[k] = (int16_t)H.chain.size();
      std::vector<int16_t> up;
      for (int a = k; a >= 0; a = parent[a]) up.push_back((int16_t)a);
      H.chain.insert(H.chain.end(), up.rbegin(), up.rend());
    }
    H.chain_start[n] = (int16_t)H.chain.size();
    for (int j = 0; j < d; ++j)
      if (jl[j].size() > 1) H.mimic_shared = 1;
  }
  H.parent.swap(parent);
  H.jidx.swap(jidx);
  H.dfs_pos.assign(n, 0);
  for (int p = 0; p < n; ++p) H.dfs_pos[H.dfs[p].x] = (int16_t)p;
  H.dfs_kj.resize(n);
  for (int p = 0; p < n; ++p) {
    const int k = H.dfs[p].x;
    const int nch = std::min(child_start[k + 1] - child_start[k], 255);
    H.dfs_kj[p] = make_int2(k | (H.dfs[p].y << 8) | ((int)H.chain_start[k] << 16),
                            (H.jidx[k] + 1) | (nch << 16) | ((int)jtype[k] << 24) |
                                ((int)rot_id[k] << 26));
  }
  H.lmeta.resize(n);
  for (int k = 0; k < n; ++k)
    H.lmeta[k] = (H.jidx[k] + 1) | ((int)jtype[k] << 16) | ((int)rot_id[k] << 24);
  // a subtree is the contiguous DFS range up to the next position at the
  // same or a smaller depth
  H.dfs_end.assign(n, (int16_t)n);
  for (int p = 0; p < n; ++p)
    for (int p2 = p + 1; p2 < n; ++p2)
      if (H.dfs[p2].y <= H.dfs[p].y) {
        H.dfs_end[H.dfs[p].x] = (int16_t)p2;
        break;
      }
  H.seg_slot.assign(3 * (size_t)n, -1);
  H.seg_slot_link.assign(3 * (size_t)n, 0);
  for (int t = 0; t < 3; ++t) plan_segments(H, t);
  H.lev_start.swap(lev_start);
  H.lev_links.swap(lev_links);
  H.child_start.swap(child_start);
  if (children.empty()) children.push_back(0);
  H.children.swap(children);
  H.jl_start.swap(jl_start);
  if (jl_links.empty()) jl_links.push_back(0);
  H.jl_links.swap(jl_links);
  H.ls_start.swap(ls_start);
  H.ls_sph.swap(ls_sph);
  H.sph_link.swap(sph_link);
  H.jtype.swap(jtype);
  H.rot_id.swap(rot_id);
  H.axis.swap(axis);
  H.Tf.swap(Tf);
  H.mimic.swap(mimic);
  H.inert.swap(inert);
  H.sp.swap(sp);
  H.grp_rad.swap(grp_rad);
  H.grp_loc.swap(grp_loc);
  H.grp_link.swap(grp_link);
  H.pairs_dev.swap(pairs_dev);
  H.bx.swap(bx);
  H.blk_pidx.swap(blk_pidx);
  return WB_OK;
}

static void fill_info(const HostPlan& H, int device, wb_robot_info* info) {
  info->n_links = H.n;
  info->dof = H.d;
  info->n_spheres = H.S;
  info->n_pairs = H.P;
  info->n_levels = H.nlev;
  info->max_level_width = H.maxw;
  info->n_pair_blocks = (int)H.bx.size();
  info->device = device;
}

extern "C" {

int wb_plan_info(const wb_tree* tree, const wb_spheres* spheres, const wb_pairs* pairs,
                 const wb_inertial* inertial, wb_robot_info* out, int32_t* sched_rounds) {
  g_err.clear();
  if (!out) return fail(WB_EINVAL, "out is NULL");
  HostPlan H;
  int rc = plan_robot(tree, spheres, pairs, inertial, H);
  if (rc != WB_OK) return rc;
  fill_info(H, -1, out);
  if (sched_rounds)
    for (int t = 0; t < 4; ++t) {
      std::vector<uint2> ent;
      int rounds = 0;
      build_schedule(4 << t, H.bx, ent, rounds);
      sched_rounds[t] = H.bx.empty() ? 0 : rounds;
    }
  return WB_OK;
}

int wb_load_robot(const wb_tree* tree, const wb_spheres* sph, const wb_pairs* pairs,
                  const wb_inertial* inertial, int device, wb_robot** out) {
  g_err.clear();
  if (!out) return fail(WB_EINVAL, "out is NULL");
  *out = nullptr;
  HostPlan H;
  int rc = plan_robot(tree, sph, pairs, inertial, H);
  if (rc != WB_OK) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(WB_EDEVICE, "device %d not available (%d devices)", device, ndev);
  }
  const int n = H.n;
  wb_robot* R = new wb_robot();
  R->device = device;
  R->n = n;
  R->S = H.S;
  DeviceGuard guard(device);
  cudaDeviceGetAttribute(&R->num_sms, cudaDevAttrMultiProcessorCount, device);

  DevRobot& D = R->dev;
  D.n = n;
  D.d = H.d;
  D.S = H.S;
  D.P = H.P;
  D.nlev = H.nlev;
  D.maxw = H.maxw;
  D.Sg = H.Sg;
  D.nblk = (int)H.bx.size();
  D.margin = (float)std::max(std::ldexp(1.0, -16), H.reach * std::ldexp(1.0, -20));
  // bound on the float rounding of the expanded squared-distance filter,
  // 128 ulp of (reach + r_max + 1 cm)^2 (see the pair stage of k_fused.cu)
  D.etol = (float)(128.0 * std::ldexp(1.0, -24) * (H.reach + H.r_max + 0.01) *
                   (H.reach + H.r_max + 0.01));
  for (int i = 0; i < 3; ++i) D.abase[i] = -H.g[i];

  Packer pk;
  pk.add_vec(H.parent, &D.parent);
  pk.add_vec(H.jtype, &D.jtype);
  pk.add_vec(H.rot_id, &D.rot_id);
  pk.add_vec(H.jidx, &D.jidx);
  pk.add_vec(H.mimic, &D.mimic);
  pk.add_vec(H.axis, &D.axis);
  pk.add_vec(H.Tf, &D.Tf);
  const size_t inert_off = pk.add_vec(H.inert, &D.inert);
  pk.add_vec(H.lev_start, &D.lev_start);
  pk.add_vec(H.lev_links, &D.lev_links);
  pk.add_vec(H.lvm, &D.lvm);
  pk.add_vec(H.dfs, &D.dfs);
  pk.add_vec(H.dfs_kj, &D.dfs_kj);
  pk.add_vec(H.lmeta, &D.lmeta);
  pk.add_vec(H.chain_start, &D.chain_start);
  pk.add_vec(H.chain, &D.chain);
  H.chain_m.resize(H.chain.size());
  for (size_t c = 0; c < H.chain.size(); ++c) {
    const int k = H.chain[c];
    H.chain_m[c] = k | ((H.jidx[k] + 1) << 8) | ((int)H.jtype[k] << 17) | ((int)H.rot_id[k] << 19);
  }
  pk.add_vec(H.chain_m, &D.chain_m);
  D.maxdepth = H.maxdepth;
  pk.add_vec(H.dfs_pos, &D.dfs_pos);
  pk.add_vec(H.dfs_end, &D.dfs_end);
  pk.add_vec(H.seg_slot, &D.seg_slot);
  pk.add_vec(H.seg_slot_link, &D.seg_slot_link);
  D.seg_ok = H.seg_ok;
  for (int t = 0; t < 3; ++t) {
    D.seg_ns[t] = H.seg_ns[t];
    for (int g = 0; g < 9; ++g) D.seg_pos[t][g] = H.seg_pos[t][g];
  }
  {
    float rmin = 0.0f;
    for (int s2 = 0; s2 < H.S; ++s2) rmin = s2 == 0 ? H.sp[s2].w : std::min(rmin, H.sp[s2].w);
    D.rmin = rmin;
    int full = 1;
    for (uint32_t x : H.bx)
      if ((x >> 16) != 0xFFFFu) full = 0;
    D.all_full = full;
    int v4 = H.S % 4 == 0 ? 1 : 0;
    for (int k = 0; k < n && v4; ++k) {
      const int e0 = H.ls_start[k], e1 = H.ls_start[k + 1];
      if ((e1 - e0) % 4) v4 = 0;
      for (int e = e0; e < e1 && v4; ++e)
        if (H.ls_sph[e] != H.ls_sph[e0 + (e - e0) / 4 * 4] + (e - e0) % 4 ||
            H.ls_sph[e0 + (e - e0) / 4 * 4] % 4)
          v4 = 0;
    }
    // then every group of 4 lies on one link (the pair stage places a group
    // from its link's pose); checked, not assumed
    for (size_t g = 0; g < H.grp_link.size() && v4; ++g)
      if (H.grp_link[g] < 0) v4 = 0;
    D.sph_vec4 = v4;
  }
  D.mimic_shared = H.mimic_shared;
  pk.add_vec(H.child_start, &D.child_start);
  pk.add_vec(H.children, &D.children);
  pk.add_vec(H.jl_start, &D.jl_start);
  pk.add_vec(H.jl_links, &D.jl_links);
  pk.add_vec(H.ls_start, &D.ls_start);
  pk.add_vec(H.ls_sph, &D.ls_sph);
  pk.add_vec(H.sp, &D.sph);
  pk.add_vec(H.sph_link, &D.sph_link);
  pk.add_vec(H.pairs_dev, &D.pairs);
  pk.add_vec(H.grp_rad, &D.grp_rad);
  pk.add_vec(H.grp_loc, &D.grp_loc);
  pk.add_vec(H.grp_link, &D.grp_link);
  pk.add_vec(H.blk_pidx, &D.blk_pidx);
  std::vector<uint2> ents[4];
  for (int t = 0; t < 4; ++t) {
    const int G = 4 << t;
    int rounds = 0;
    build_schedule(G, H.bx, ents[t], rounds);
    R->sched[t].G = G;
    R->sched[t].rounds = H.bx.empty() ? 0 : rounds;
    pk.add_vec(ents[t], &R->sched[t].ent);
  }
  std::vector<uint2> ent32(ents[3]);
  for (auto& e : ent32) {
    const uint32_t gi = e.x & 0xFF, gj = (e.x >> 8) & 0xFF, mask = e.x >> 16;
    e = uint2{(16u * gi) | ((16u * gj) << 16), (mask << 16) | (e.y & 0xFFFF)};
  }
  R->sched32.rounds = R->sched[3].rounds;
  pk.add_vec(ent32, &R->sched32.ent);
  cudaError_t e = cudaMalloc(&R->dmem, pk.host.size());
  if (e != cudaSuccess) {
    delete R;
    return cuda_fail(e, "cudaMalloc(robot)");
  }
  R->dbytes = pk.host.size();
  e = cudaMemcpy(R->dmem, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(R->dmem);
    delete R;
    return cuda_fail(e, "cudaMemcpy(robot)");
  }
  for (auto& it : pk.items) *it.slot = static_cast<char*>(R->dmem) + it.off;
  R->d_inert = reinterpret_cast<float*>(static_cast<char*>(R->dmem) + inert_off);
  e = cudaMallocHost(reinterpret_cast<void**>(&R->h_stage), H.inert.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->stage_evt, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    wb_free_robot(R);
    return cuda_fail(e, "robot staging buffer");
  }
  fill_info(H, device, &R->info);
  *out = R;
  return WB_OK;
}

int wb_robot_info_get(const wb_robot* robot, wb_robot_info* out) {
  if (!robot || !out) return fail(WB_EINVAL, "NULL argument");
  *out = robot->info;
  return WB_OK;
}

int wb_set_inertials(wb_robot* robot, const wb_inertial* inertial, void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  std::vector<float> inert;
  int rc = compact_inertia(inertial, robot->n, inert);
  if (rc != WB_OK) return rc;
  DeviceGuard guard(robot->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (robot->stage_pending) {
    cudaError_t e = cudaEventSynchronize(robot->stage_evt);
    if (e != cudaSuccess) return cuda_fail(e, "wait for previous inertia upload");
  }
  std::memcpy(robot->h_stage, inert.data(), inert.size() * sizeof(float));
  cudaError_t e = cudaMemcpyAsync(robot->d_inert, robot->h_stage, inert.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "inertia upload");
  e = cudaEventRecord(robot->stage_evt, s);
  if (e != cudaSuccess) return cuda_fail(e, "inertia upload event");
  robot->stage_pending = true;
  return WB_OK;
}

void wb_free_robot(wb_robot* robot) {
  if (!robot) return;
  {
    DeviceGuard guard(robot->device);
    if (robot->stage_pending) cudaEventSynchronize(robot->stage_evt);
    if (robot->stage_evt) cudaEventDestroy(robot->stage_evt);
    if (robot->h_stage) cudaFreeHost(robot->h_stage);
    if (robot->dmem) cudaFree(robot->dmem);
  }
  delete robot;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
static int check_ptr(const wb_robot* R, const void* p, const char* name, bool required) {
  if (!p) return required ? fail(WB_EINVAL, "%s is NULL", name) : WB_OK;
  if (reinterpret_cast<uintptr_t>(p) & 15u)
    return fail(WB_EINVAL, "%s is not 16-byte aligned", name);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(WB_EDEVICE, "%s: not a CUDA pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(WB_EDEVICE, "%s is not device memory", name);
  if (at.type == cudaMemoryTypeDevice && at.device != R->device)
    return fail(WB_EDEVICE, "%s lives on device %d, robot on device %d", name, at.device,
                R->device);
  return WB_OK;
}

static int default_G(const DevRobot& r) { return (r.n >= 24 || r.P >= 2048) ? 32 : 8; }

// Pick configurations per CTA and grid for a fused launch.
static int fused_shape(const wb_robot* R, bool fwd, bool bits, const wb_tune* t, int64_t B,
                       FusedShape& sh) {
  const DevRobot& D = R->dev;
  int G = (t && t->lanes_per_config) ? t->lanes_per_config : default_G(D);
  if (sched_slot(G) < 0) return fail(WB_EINVAL, "lanes_per_config must be 4, 8, 16 or 32");
  const size_t per = fwd ? fused_fwd_smem_per_config(D, G, bits) : fused_bwd_smem_per_config(D, G);
  const size_t cta = fused_cta_smem(D);
  const int step = 32 / G;  // configurations per warp
  int cpb = (t && t->configs_per_block) ? t->configs_per_block : 0;
  if (cpb) {
    if (cpb % step) return fail(WB_EINVAL, "configs_per_block must be a multiple of %d", step);
    if (cpb * G > 256) return fail(WB_EINVAL, "configs_per_block * lanes must be <= 256");
  } else {
    // most resident warps per SM: try every CTA size, keep the best
    cpb = step;
    int best_warps = -1;
    for (int c = step; c * G <= 256; c += step) {
      const size_t sm = cta + per * c;
      if (sm > 227 * 1024) break;
      int nb = 0;
      cudaError_t e = fwd ? fused_fwd_max_blocks_per_sm(G, c, sm, &nb)
                          : fused_bwd_max_blocks_per_sm(G, c, sm, &nb);
      if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
      const int warps = nb * c * G / 32;
      if (warps > best_warps) {
        best_warps = warps;
        cpb = c;
      }
    }
  }
  const size_t smem = cta + per * cpb;
  if (smem > 227 * 1024)
    return fail(WB_ETOOBIG, "robot needs %zu bytes of shared memory per CTA", smem);
  int bps = (t && t->blocks_per_sm) ? t->blocks_per_sm : 0;
  if (!bps) {
    cudaError_t e = fwd ? fused_fwd_max_blocks_per_sm(G, cpb, smem, &bps)
                        : fused_bwd_max_blocks_per_sm(G, cpb, smem, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (bps < 1) return fail(WB_ETOOBIG, "fused kernel does not fit on an SM");
  }
  const int64_t ntiles = (B + cpb - 1) / cpb;
  sh.G = G;
  sh.cpb = cpb;
  sh.smem = smem;
  sh.grid = (int)std::min<int64_t>(ntiles, (int64_t)bps * R->num_sms);
  return WB_OK;
}

static bool plain_fits(const DevRobot& D) { return D.n <= 64 && D.S <= 256; }

// The one-warp-per-configuration kernels (pair map-reduce, summed hinge,
// kinematics) keep a per-warp workspace in shared memory; a block takes the
// most warps, up to 8, whose workspaces fit in one CTA's shared memory
// (0: not even one fits).
constexpr size_t kMaxBlockSmem = 227 * 1024;
static int warps_that_fit(size_t fixed_bytes, size_t per_warp_bytes) {
  for (int w = 8; w >= 1; --w)
    if (fixed_bytes + per_warp_bytes * w <= kMaxBlockSmem) return w;
  return 0;
}
// Warps per block of the pair kernel (wb_tune.blocks_per_sm for TREE): the
// tuned count; else, for the culled kernel, the count in 4..8 (of those whose
// workspaces fit a block) whose blocks keep the most warps resident on an SM,
// the fewest on a tie -- smaller blocks let the persistent grid deal its
// configurations in finer pieces; for the full map-reduce (TREE_NOCULL) the
// most that fit.  Measured on the 48-DoF humanoid at 32768 configurations,
// culled: 4 warps (7 blocks, 28 warps an SM) 0.176 ms, 7 warps (4 blocks)
// 0.183 ms, 8 warps (3 blocks, 24 warps) 0.185 ms; the full map-reduce
// 0.33 ms at 8 warps, 0.40 ms at 4.
static int pair_warps(wb_robot* R, bool bits, const wb_tune* tune, bool cull = true) {
  if (tune && tune->blocks_per_sm) return tune->blocks_per_sm;
  const DevRobot& D = R->dev;
  const size_t one = pair_block_smem(D, 1, bits), none = pair_block_smem(D, 0, bits);
  const int most = warps_that_fit(none, one - none);
  if (!cull) return most;
  std::atomic<int>& cached = R->pair_warps_default[bits ? 1 : 0];
  if (const int c = cached.load(std::memory_order_relaxed)) return c;
  int best = most, best_res = -1;
  for (int w = 4; w <= most; ++w) {
    int bps = 0;
    if (pair_max_blocks_per_sm(D, w, bits, &bps) != cudaSuccess) {
      cudaGetLastError();
      best = most;
      break;
    }
    if (w * bps > best_res) {
      best_res = w * bps;
      best = w;
    }
  }
  cached.store(best, std::memory_order_relaxed);
  return best;
}

// Segments of the sweep kernels (wb_tune.lanes_per_config for TREE): 1, 2, 4
// or 8; 0 = the fewest of the robot's plans that give about 12 warps per SM --
// measured on the 48-DoF humanoid at 32768 configurations: both passes best
// at 2 segments (the register copies of the stack top make each warp
// faster, so fewer segments suffice), 8 slower than 1.
static int tree_segments(const wb_robot* R, const wb_tune* tune, int64_t B, int threads,
                         bool fwd, int* out) {
  const int req = tune ? tune->lanes_per_config : 0;
  const int ok = R->dev.seg_ok;
  int G = 1;
  if (req > 0) {
    const int t = req == 2 ? 0 : req == 4 ? 1 : req == 8 ? 2 : -1;
    if (req != 1 && t < 0) return fail(WB_EINVAL, "tree segments must be 1, 2, 4 or 8");
    if (t >= 0 && !(ok >> t & 1))
      return fail(WB_EINVAL, "no %d-segment sweep for this robot (fewer links, or a joint "
                  "driving several links)", req);
    G = req;
  } else {
    const int64_t warps = (B + 31) / 32;
    const int64_t target = 12LL * R->num_sms;
    for (int t = 0; t < 3 && warps * G < target; ++t)
      if (ok >> t & 1) G = 2 << t;
  }
  if (G == 1 && threads > 256)
    return fail(WB_EINVAL, "one-segment sweeps take at most 256 threads per block");
  if (G > 1 && tree_seg_smem(R->dev, G, threads, fwd, !fwd) +
                       (fwd ? 0 : grad_slot_smem(G, threads)) >
                   227 * 1024)
    return fail(WB_ETOOBIG, "segmented sweep needs too much shared memory");
  *out = G;
  return WB_OK;
}

extern "C" {

int wb_eval(wb_robot* robot, int64_t B, const float* q, const float* qd, const float* qdd,
            float* link_pose, float* sphere, float* d_min, int32_t* worst_pair, float* tau,
            uint32_t* pair_bits, const wb_tune* tune, void* stream) {
  return wb_eval_ext(robot, B, q, qd, qdd, nullptr, link_pose, sphere, d_min, worst_pair, tau,
                     pair_bits, tune, stream);
}

int wb_eval_ext(wb_robot* robot, int64_t B, const float* q, const float* qd, const float* qdd,
                const float* f_ext, float* link_pose, float* sphere, float* d_min,
                int32_t* worst_pair, float* tau, uint32_t* pair_bits, const wb_tune* tune,
                void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (B < 0) return fail(WB_EINVAL, "B < 0");
  if (B == 0) return WB_OK;
  if (B > (int64_t)1 << 40) return fail(WB_EINVAL, "B too large");
  int rc;
  if ((rc = check_ptr(robot, q, "q", true))) return rc;
  if ((rc = check_ptr(robot, qd, "qd", tau != nullptr))) return rc;
  if ((rc = check_ptr(robot, qdd, "qdd", tau != nullptr))) return rc;
  if ((rc = check_ptr(robot, link_pose, "link_pose", false))) return rc;
  if ((rc = check_ptr(robot, sphere, "sphere", false))) return rc;
  if ((rc = check_ptr(robot, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(robot, worst_pair, "worst_pair", d_min != nullptr))) return rc;
  if ((rc = check_ptr(robot, tau, "tau", false))) return rc;
  if ((rc = check_ptr(robot, pair_bits, "pair_bits", false))) return rc;
  if ((rc = check_ptr(robot, f_ext, "f_ext", false))) return rc;
  if (!d_min && worst_pair) return fail(WB_EINVAL, "worst_pair without d_min");
  DeviceGuard guard(robot->device);
  FwdArgs a{B, q, qd, qdd, link_pose, sphere, d_min, worst_pair, tau, pair_bits};
  a.fext = tau ? f_ext : nullptr;
  int kernel = tune ? tune->kernel : WB_KERNEL_AUTO;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool pairs_wanted = d_min || sphere || pair_bits;
  const bool tree_ok = robot->dev.maxdepth <= tree_max_depth();
  if (kernel == WB_KERNEL_AUTO)
    kernel = (tree_ok && (link_pose || !pairs_wanted)) ? WB_KERNEL_TREE : WB_KERNEL_FUSED;
  cudaError_t e;
  const bool cull = kernel != WB_KERNEL_TREE_NOCULL;
  if (kernel == WB_KERNEL_TREE_NOCULL) kernel = WB_KERNEL_TREE;
  if (kernel == WB_KERNEL_PLAIN) {
    if (!plain_fits(robot->dev))
      return fail(WB_ETOOBIG, "plain kernel supports at most 64 links and 256 spheres");
    e = launch_plain_fwd(robot->dev, a, 128, s);
  } else if (kernel == WB_KERNEL_TREE) {
    if (!tree_ok) return fail(WB_ETOOBIG, "tree deeper than %d levels", tree_max_depth());
    if (pairs_wanted && !link_pose)
      return fail(WB_EINVAL, "the tree kernel needs link_pose when spheres or pairs are wanted");
    const int tpb = (tune && tune->configs_per_block) ? tune->configs_per_block : 128;
    if (tpb < 32 || tpb > 512 || tpb % 32)
      return fail(WB_EINVAL, "tree threads per block must be a multiple of 32 in [32, 512]");
    const int warps = pair_warps(robot, pair_bits != nullptr, tune, cull);
    if (tune && tune->blocks_per_sm && (warps < 1 || warps > 8))
      return fail(WB_EINVAL, "pair warps per block must be in [1, 8]");
    if (pairs_wanted && warps == 0) return fail(WB_ETOOBIG, "pair kernel does not fit on an SM");
    if (pairs_wanted && pair_block_smem(robot->dev, warps, pair_bits != nullptr) > kMaxBlockSmem)
      return fail(WB_ETOOBIG, "%d pair warps per block need too much shared memory", warps);
    int G = 1;
    if ((rc = tree_segments(robot, tune, B, tpb, true, &G))) return rc;
    e = launch_tree_fwd(robot->dev, a, tpb, G, s);
    if (e == cudaSuccess && pairs_wanted) {
      int bps = 0;
      e = pair_max_blocks_per_sm(robot->dev, warps, pair_bits != nullptr, &bps);
      if (e == cudaSuccess) {
        if (bps < 1) return fail(WB_ETOOBIG, "pair kernel does not fit on an SM");
        const int64_t need = (B + warps - 1) / warps;
        const int grid = (int)std::min<int64_t>(need, (int64_t)bps * robot->num_sms);
        e = launch_pair(robot->dev, robot->sched32, a, grid, warps, s, cull);
      }
    }
  } else if (kernel == WB_KERNEL_FUSED) {
    if (a.fext) return fail(WB_EINVAL, "the fused kernels take no external forces");
    FusedShape sh;
    if ((rc = fused_shape(robot, true, pair_bits != nullptr, tune, B, sh))) return rc;
    e = launch_fused_fwd(robot->dev, robot->sched[sched_slot(sh.G)], a, sh, s);
  } else {
    return fail(WB_EINVAL, "unknown kernel %d", kernel);
  }
  if (e != cudaSuccess) return cuda_fail(e, "wb_eval launch");
  return WB_OK;
}

int wb_self_collision(wb_robot* robot, int64_t B, const float* link_pose, float* sphere,
                      float* d_min, int32_t* worst_pair, uint32_t* pair_bits, void* stream) {
  return wb_self_collision_tuned(robot, B, link_pose, sphere, d_min, worst_pair, pair_bits,
                                 nullptr, stream);
}

int wb_self_collision_tuned(wb_robot* robot, int64_t B, const float* link_pose, float* sphere,
                            float* d_min, int32_t* worst_pair, uint32_t* pair_bits,
                            const wb_tune* tune, void* stream) {
  return wb_self_collision_dir(robot, B, link_pose, sphere, d_min, worst_pair, nullptr, pair_bits,
                               tune, stream);
}

int wb_self_collision_dir(wb_robot* robot, int64_t B, const float* link_pose, float* sphere,
                          float* d_min, int32_t* worst_pair, float* worst_diff,
                          uint32_t* pair_bits, const wb_tune* tune, void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (B < 0) return fail(WB_EINVAL, "B < 0");
  if (B == 0) return WB_OK;
  int rc;
  if ((rc = check_ptr(robot, link_pose, "link_pose", true))) return rc;
  if ((rc = check_ptr(robot, sphere, "sphere", false))) return rc;
  if ((rc = check_ptr(robot, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(robot, worst_pair, "worst_pair", d_min != nullptr))) return rc;
  if ((rc = check_ptr(robot, worst_diff, "worst_diff", false))) return rc;
  if ((rc = check_ptr(robot, pair_bits, "pair_bits", false))) return rc;
  if (!d_min && worst_pair) return fail(WB_EINVAL, "worst_pair without d_min");
  if (!d_min && worst_diff) return fail(WB_EINVAL, "worst_diff without d_min");
  if (!d_min && !sphere && !pair_bits) return WB_OK;
  DeviceGuard guard(robot->device);
  FwdArgs a{B, nullptr, nullptr, nullptr, const_cast<float*>(link_pose), sphere, d_min,
            worst_pair, nullptr, pair_bits};
  a.wdiff = worst_diff;
  const int kernel = tune ? tune->kernel : WB_KERNEL_AUTO;
  if (kernel != WB_KERNEL_AUTO && kernel != WB_KERNEL_TREE && kernel != WB_KERNEL_TREE_NOCULL)
    return fail(WB_EINVAL, "the pair kernel takes TREE (culled) or TREE_NOCULL");
  const int warps = pair_warps(robot, pair_bits != nullptr, tune, kernel != WB_KERNEL_TREE_NOCULL);
  if (tune && tune->blocks_per_sm && (warps < 1 || warps > 8))
    return fail(WB_EINVAL, "pair warps per block must be in [1, 8]");
  if (warps == 0) return fail(WB_ETOOBIG, "pair kernel does not fit on an SM");
  if (pair_block_smem(robot->dev, warps, pair_bits != nullptr) > kMaxBlockSmem)
    return fail(WB_ETOOBIG, "%d pair warps per block need too much shared memory", warps);
  int bps = 0;
  cudaError_t e = pair_max_blocks_per_sm(robot->dev, warps, pair_bits != nullptr, &bps);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(WB_ETOOBIG, "pair kernel does not fit on an SM");
  const int64_t need = (B + warps - 1) / warps;
  const int grid = (int)std::min<int64_t>(need, (int64_t)bps * robot->num_sms);
  e = launch_pair(robot->dev, robot->sched32, a, grid, warps, static_cast<cudaStream_t>(stream),
                  kernel != WB_KERNEL_TREE_NOCULL);
  if (e != cudaSuccess) return cuda_fail(e, "wb_self_collision launch");
  return WB_OK;
}

int wb_kinematics(wb_robot* robot, int64_t B, const float* link_pose, int32_t n_targets,
                  const int32_t* targets, float* jac, float* com, float* jac_com, void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (B < 0) return fail(WB_EINVAL, "B < 0");
  if (n_targets < 0 || n_targets > KIN_MAX_TARGETS)
    return fail(WB_EINVAL, "n_targets must be in [0, %d]", KIN_MAX_TARGETS);
  if (n_targets > 0 && !targets) return fail(WB_EINVAL, "targets is NULL");
  KinArgs a{};
  for (int t = 0; t < n_targets; ++t) {
    if (targets[t] < 0 || targets[t] >= robot->dev.n)
      return fail(WB_ERANGE, "target %d = link %d out of range", t, targets[t]);
    a.targets[t] = targets[t];
  }
  if (jac && n_targets == 0) jac = nullptr;
  if (B == 0 || (!jac && !com && !jac_com)) return WB_OK;
  int rc;
  if ((rc = check_ptr(robot, link_pose, "link_pose", true))) return rc;
  if ((rc = check_ptr(robot, jac, "jac", false))) return rc;
  if ((rc = check_ptr(robot, com, "com", false))) return rc;
  if ((rc = check_ptr(robot, jac_com, "jac_com", false))) return rc;
  DeviceGuard guard(robot->device);
  const int warps = warps_that_fit(0, kin_smem_per_warp(robot->dev));
  if (warps == 0) return fail(WB_ETOOBIG, "kinematics kernel does not fit on an SM");
  int bps = 0;
  cudaError_t e = kin_max_blocks_per_sm(robot->dev, warps, &bps);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(WB_ETOOBIG, "kinematics kernel does not fit on an SM");
  const int64_t need = (B + warps - 1) / warps;
  const int grid = (int)std::min<int64_t>(need, (int64_t)bps * robot->num_sms);
  a.B = B;
  a.pose = link_pose;
  a.nt = n_targets;
  a.jac = jac;
  a.com = com;
  a.jac_com = jac_com;
  e = launch_kin(robot->dev, a, grid, warps, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_kinematics launch");
  return WB_OK;
}

int wb_self_collision_hinge(wb_robot* robot, int64_t B, const float* link_pose, float eta,
                            float w, float* cost, float* g_sphere, void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (B < 0) return fail(WB_EINVAL, "B < 0");
  if (!std::isfinite(eta) || !std::isfinite(w)) return fail(WB_EINVAL, "eta and w must be finite");
  if (B == 0 || (!cost && !g_sphere)) return WB_OK;
  int rc;
  if ((rc = check_ptr(robot, link_pose, "link_pose", true))) return rc;
  if ((rc = check_ptr(robot, cost, "cost", false))) return rc;
  if ((rc = check_ptr(robot, g_sphere, "g_sphere", false))) return rc;
  DeviceGuard guard(robot->device);
  const int warps = warps_that_fit(hinge_smem_fixed(robot->dev), hinge_smem_per_warp(robot->dev));
  if (warps == 0) return fail(WB_ETOOBIG, "hinge kernel does not fit on an SM");
  int bps = 0;
  cudaError_t e = hinge_max_blocks_per_sm(robot->dev, warps, &bps);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(WB_ETOOBIG, "hinge kernel does not fit on an SM");
  const int64_t need = (B + warps - 1) / warps;
  const int grid = (int)std::min<int64_t>(need, (int64_t)bps * robot->num_sms);
  HingeArgs a{B, link_pose, eta, w, cost, g_sphere};
  e = launch_hinge(robot->dev, robot->sched32, a, grid, warps, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_self_collision_hinge launch");
  return WB_OK;
}

int wb_eval_backward(wb_robot* robot, int64_t B, const float* q, const float* qd,
                     const float* qdd, const int32_t* worst_pair, const float* g_pose,
                     const float* g_sphere, const float* g_dmin, const float* g_tau, float* gq,
                     float* gqd, float* gqdd, const wb_tune* tune, void* stream) {
  return wb_eval_backward_ext(robot, B, q, qd, qdd, nullptr, worst_pair, g_pose, g_sphere,
                              g_dmin, g_tau, gq, gqd, gqdd, nullptr, tune, stream);
}

int wb_eval_backward_ext(wb_robot* robot, int64_t B, const float* q, const float* qd,
                         const float* qdd, const float* f_ext, const int32_t* worst_pair,
                         const float* g_pose, const float* g_sphere, const float* g_dmin,
                         const float* g_tau, float* gq, float* gqd, float* gqdd, float* g_fext,
                         const wb_tune* tune, void* stream) {
  return wb_eval_backward_dir(robot, B, q, qd, qdd, f_ext, worst_pair, nullptr, g_pose, g_sphere,
                              g_dmin, g_tau, gq, gqd, gqdd, g_fext, tune, stream);
}

int wb_eval_backward_dir(wb_robot* robot, int64_t B, const float* q, const float* qd,
                         const float* qdd, const float* f_ext, const int32_t* worst_pair,
                         const float* worst_diff, const float* g_pose, const float* g_sphere,
                         const float* g_dmin, const float* g_tau, float* gq, float* gqd,
                         float* gqdd, float* g_fext, const wb_tune* tune, void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (B < 0) return fail(WB_EINVAL, "B < 0");
  if (B == 0) return WB_OK;
  if (B > (int64_t)1 << 40) return fail(WB_EINVAL, "B too large");
  int rc;
  if ((rc = check_ptr(robot, q, "q", true))) return rc;
  if ((rc = check_ptr(robot, qd, "qd", true))) return rc;
  if ((rc = check_ptr(robot, qdd, "qdd", true))) return rc;
  if ((rc = check_ptr(robot, worst_pair, "worst_pair", g_dmin != nullptr))) return rc;
  if ((rc = check_ptr(robot, g_pose, "g_pose", false))) return rc;
  if ((rc = check_ptr(robot, g_sphere, "g_sphere", false))) return rc;
  if ((rc = check_ptr(robot, g_dmin, "g_dmin", false))) return rc;
  if ((rc = check_ptr(robot, g_tau, "g_tau", false))) return rc;
  if ((rc = check_ptr(robot, gq, "gq", true))) return rc;
  if ((rc = check_ptr(robot, gqd, "gqd", true))) return rc;
  if ((rc = check_ptr(robot, gqdd, "gqdd", true))) return rc;
  if ((rc = check_ptr(robot, f_ext, "f_ext", false))) return rc;
  if ((rc = check_ptr(robot, g_fext, "g_fext", false))) return rc;
  if ((rc = check_ptr(robot, worst_diff, "worst_diff", false))) return rc;
  DeviceGuard guard(robot->device);
  BwdArgs a{B, q, qd, qdd, worst_pair, g_pose, g_sphere, g_dmin, g_tau, gq, gqd, gqdd};
  a.fext = f_ext;
  a.g_fext = g_fext;
  a.wdiff = worst_diff;
  if (g_fext && !g_tau) {  // nothing depends on the external forces but tau
    cudaError_t e0 = cudaMemsetAsync(g_fext, 0, sizeof(float) * 6 * robot->dev.n * B,
                                     static_cast<cudaStream_t>(stream));
    if (e0 != cudaSuccess) return cuda_fail(e0, "g_fext clear");
    a.g_fext = nullptr;
  }
  int kernel = tune ? tune->kernel : WB_KERNEL_AUTO;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tree_ok = robot->dev.maxdepth <= tree_max_depth();
  if (kernel == WB_KERNEL_AUTO) kernel = tree_ok ? WB_KERNEL_TREE : WB_KERNEL_FUSED;
  if (kernel == WB_KERNEL_TREE_NOCULL) kernel = WB_KERNEL_TREE;  // no pair stage here
  cudaError_t e;
  if (kernel == WB_KERNEL_PLAIN) {
    if (!plain_fits(robot->dev))
      return fail(WB_ETOOBIG, "plain kernel supports at most 64 links and 256 spheres");
    e = launch_plain_bwd(robot->dev, a, 128, s);
  } else if (kernel == WB_KERNEL_TREE) {
    if (!tree_ok) return fail(WB_ETOOBIG, "tree deeper than %d levels", tree_max_depth());
    const int tpb = (tune && tune->configs_per_block) ? tune->configs_per_block : 128;
    if (tpb < 32 || tpb > 512 || tpb % 32)
      return fail(WB_EINVAL, "tree threads per block must be a multiple of 32 in [32, 512]");
    int G = 1;
    if ((rc = tree_segments(robot, tune, B, tpb, false, &G))) return rc;
    e = launch_tree_bwd(robot->dev, a, tpb, G, s);
  } else if (kernel == WB_KERNEL_FUSED) {
    if (a.fext || a.g_fext) return fail(WB_EINVAL, "the fused kernels take no external forces");
    FusedShape sh;
    if ((rc = fused_shape(robot, false, false, tune, B, sh))) return rc;
    e = launch_fused_bwd(robot->dev, a, sh, s);
  } else {
    return fail(WB_EINVAL, "unknown kernel %d", kernel);
  }
  if (e != cudaSuccess) return cuda_fail(e, "wb_eval_backward launch");
  return WB_OK;
}

// the spline source of the _spline entry points: validated, on the robot's device
static int check_spline_src(const wb_robot* robot, const wb_spline* sp, SplineArgs* out,
                            int64_t* B) {
  if (!sp) return fail(WB_EINVAL, "spline is NULL");
  if (sp->n_traj < 0) return fail(WB_EINVAL, "n_traj < 0");
  if (sp->K < 4 || sp->K > 4096)
    return fail(WB_EINVAL, "K = %d outside [4, 4096] (a cubic B-spline needs 4 control points)",
                sp->K);
  if (sp->T < 2 || sp->T > 4096) return fail(WB_EINVAL, "T = %d outside [2, 4096]", sp->T);
  if (!(sp->dt > 0.0f) || !std::isfinite(sp->dt)) return fail(WB_EINVAL, "dt must be positive");
  if (sp->n_traj * sp->T > ((int64_t)1 << 40)) return fail(WB_EINVAL, "too many samples");
  int rc;
  if ((rc = check_ptr(robot, sp->U, "U", sp->n_traj > 0))) return rc;
  out->U = sp->U;
  out->K = sp->K;
  out->T = sp->T;
  out->dt = sp->dt;
  *B = sp->n_traj * sp->T;
  return WB_OK;
}

int wb_eval_spline(wb_robot* robot, const wb_spline* spline, float* link_pose, float* sphere,
                   float* d_min, int32_t* worst_pair, float* tau, const wb_tune* tune,
                   void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  SplineArgs sp;
  int64_t B = 0;
  int rc;
  if ((rc = check_spline_src(robot, spline, &sp, &B))) return rc;
  if (B == 0) return WB_OK;
  const bool pairs_wanted = d_min || sphere;
  if (pairs_wanted && !link_pose) return fail(WB_EINVAL, "spheres or pairs need link_pose");
  if (d_min && !worst_pair) return fail(WB_EINVAL, "d_min without worst_pair");
  if ((rc = check_ptr(robot, link_pose, "link_pose", false))) return rc;
  if ((rc = check_ptr(robot, sphere, "sphere", false))) return rc;
  if ((rc = check_ptr(robot, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(robot, worst_pair, "worst_pair", false))) return rc;
  if ((rc = check_ptr(robot, tau, "tau", false))) return rc;
  int kernel = tune ? tune->kernel : WB_KERNEL_AUTO;
  if (kernel != WB_KERNEL_AUTO && kernel != WB_KERNEL_TREE && kernel != WB_KERNEL_TREE_NOCULL)
    return fail(WB_EINVAL, "the spline sweeps are tree kernels (kernel AUTO, TREE or TREE_NOCULL)");
  if (robot->dev.maxdepth > tree_max_depth())
    return fail(WB_ETOOBIG, "tree deeper than %d levels", tree_max_depth());
  DeviceGuard guard(robot->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FwdArgs a{B, nullptr, nullptr, nullptr, link_pose, sphere, d_min, worst_pair, tau, nullptr};
  const int tpb = (tune && tune->configs_per_block) ? tune->configs_per_block : 128;
  if (tpb < 32 || tpb > 512 || tpb % 32)
    return fail(WB_EINVAL, "tree threads per block must be a multiple of 32 in [32, 512]");
  int G = 1;
  if ((rc = tree_segments(robot, tune, B, tpb, true, &G))) return rc;
  cudaError_t e = launch_tree_fwd_spline(robot->dev, a, sp, tpb, G, s);
  if (e == cudaSuccess && pairs_wanted) {
    const int warps = pair_warps(robot, false, tune, kernel != WB_KERNEL_TREE_NOCULL);
    if (warps < 1 || warps > 8) return fail(WB_ETOOBIG, "pair kernel does not fit on an SM");
    int bps = 0;
    e = pair_max_blocks_per_sm(robot->dev, warps, false, &bps);
    if (e == cudaSuccess) {
      if (bps < 1) return fail(WB_ETOOBIG, "pair kernel does not fit on an SM");
      const int64_t need = (B + warps - 1) / warps;
      const int grid = (int)std::min<int64_t>(need, (int64_t)bps * robot->num_sms);
      e = launch_pair(robot->dev, robot->sched32, a, grid, warps, s,
                      kernel != WB_KERNEL_TREE_NOCULL);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "wb_eval_spline launch");
  return WB_OK;
}

int wb_eval_backward_spline_cost(wb_robot* robot, const wb_spline* spline,
                                 const int32_t* worst_pair, const float* g_pose,
                                 const float* g_sphere, const float* tau, const float* d_min,
                                 const float* tau_lo, const float* tau_hi,
                                 const wb_cost_weights* w, float* cost, float* gq, float* gqd,
                                 float* gqdd, const wb_tune* tune, void* stream) {
  return wb_eval_backward_spline_cost_dir(robot, spline, worst_pair, nullptr, g_pose, g_sphere,
                                          tau, d_min, tau_lo, tau_hi, w, cost, gq, gqd, gqdd,
                                          tune, stream);
}

int wb_eval_backward_spline_cost_dir(wb_robot* robot, const wb_spline* spline,
                                     const int32_t* worst_pair, const float* worst_diff,
                                     const float* g_pose, const float* g_sphere,
                                     const float* tau, const float* d_min, const float* tau_lo,
                                     const float* tau_hi, const wb_cost_weights* w, float* cost,
                                     float* gq, float* gqd, float* gqdd, const wb_tune* tune,
                                     void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (!w) return fail(WB_EINVAL, "weights are NULL");
  const wb_cost_weights W = *w;
  if (!std::isfinite(W.collision) || !std::isfinite(W.smooth) || !std::isfinite(W.length) ||
      !std::isfinite(W.energy) || !std::isfinite(W.dt) || !(W.dt > 0.0f) ||
      !std::isfinite(W.energy * W.dt * W.dt))
    return fail(WB_EINVAL, "weights must be finite and dt > 0");
  SplineArgs sp;
  int64_t B = 0;
  int rc;
  if ((rc = check_spline_src(robot, spline, &sp, &B))) return rc;
  if (B == 0) return WB_OK;
  if (robot->dev.mimic_shared)
    return fail(WB_EINVAL, "the fused cost needs one link per joint (no shared mimic joints)");
  if ((rc = check_ptr(robot, tau, "tau", true))) return rc;
  if ((rc = check_ptr(robot, tau_lo, "tau_lo", true))) return rc;
  if ((rc = check_ptr(robot, tau_hi, "tau_hi", true))) return rc;
  if ((rc = check_ptr(robot, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(robot, worst_pair, "worst_pair", d_min != nullptr))) return rc;
  if ((rc = check_ptr(robot, g_pose, "g_pose", false))) return rc;
  if ((rc = check_ptr(robot, g_sphere, "g_sphere", false))) return rc;
  if ((rc = check_ptr(robot, cost, "cost", false))) return rc;
  if ((rc = check_ptr(robot, gq, "gq", true))) return rc;
  if ((rc = check_ptr(robot, gqd, "gqd", true))) return rc;
  if ((rc = check_ptr(robot, gqdd, "gqdd", true))) return rc;
  if ((rc = check_ptr(robot, worst_diff, "worst_diff", false))) return rc;
  int kernel = tune ? tune->kernel : WB_KERNEL_AUTO;
  if (kernel == WB_KERNEL_TREE_NOCULL) kernel = WB_KERNEL_TREE;
  if (kernel != WB_KERNEL_AUTO && kernel != WB_KERNEL_TREE)
    return fail(WB_EINVAL, "the fused cost runs in the tree kernels (kernel AUTO or TREE)");
  if (robot->dev.maxdepth > tree_max_depth())
    return fail(WB_ETOOBIG, "tree deeper than %d levels", tree_max_depth());
  DeviceGuard guard(robot->device);
  BwdArgs a{B, nullptr, nullptr, nullptr, worst_pair, g_pose, g_sphere, nullptr, nullptr,
            gq, gqd, gqdd};
  a.wdiff = worst_diff;
  FusedCost fc;
  fc.tau = tau;
  fc.d_min = d_min;
  fc.lo = tau_lo;
  fc.hi = tau_hi;
  fc.w = W.collision;
  fc.smooth = W.smooth;
  fc.length = W.length;
  fc.e = W.energy * W.dt * W.dt;
  fc.cost = cost;
  const int tpb = (tune && tune->configs_per_block) ? tune->configs_per_block : 128;
  if (tpb < 32 || tpb > 512 || tpb % 32)
    return fail(WB_EINVAL, "tree threads per block must be a multiple of 32 in [32, 512]");
  int G = 1;
  if ((rc = tree_segments(robot, tune, B, tpb, false, &G))) return rc;
  const cudaError_t e = launch_tree_bwd_spline_cost(robot->dev, a, fc, sp, tpb, G,
                                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_eval_backward_spline_cost launch");
  return WB_OK;
}

int wb_eval_backward_cost(wb_robot* robot, int64_t B, const float* q, const float* qd,
                          const float* qdd, const int32_t* worst_pair, const float* g_pose,
                          const float* g_sphere, const float* tau, const float* d_min,
                          const float* tau_lo, const float* tau_hi, const wb_cost_weights* w,
                          float* cost, float* gq, float* gqd, float* gqdd, const wb_tune* tune,
                          void* stream) {
  return wb_eval_backward_cost_dir(robot, B, q, qd, qdd, worst_pair, nullptr, g_pose, g_sphere,
                                   tau, d_min, tau_lo, tau_hi, w, cost, gq, gqd, gqdd, tune,
                                   stream);
}

int wb_eval_backward_cost_dir(wb_robot* robot, int64_t B, const float* q, const float* qd,
                              const float* qdd, const int32_t* worst_pair,
                              const float* worst_diff, const float* g_pose,
                              const float* g_sphere, const float* tau, const float* d_min,
                              const float* tau_lo, const float* tau_hi, const wb_cost_weights* w,
                              float* cost, float* gq, float* gqd, float* gqdd,
                              const wb_tune* tune, void* stream) {
  g_err.clear();
  if (!robot) return fail(WB_EINVAL, "robot is NULL");
  if (!w) return fail(WB_EINVAL, "weights are NULL");
  const wb_cost_weights W = *w;
  if (!std::isfinite(W.collision) || !std::isfinite(W.smooth) || !std::isfinite(W.length) ||
      !std::isfinite(W.energy) || !std::isfinite(W.dt) || !(W.dt > 0.0f) ||
      !std::isfinite(W.energy * W.dt * W.dt))
    return fail(WB_EINVAL, "weights must be finite and dt > 0");
  if (B < 0) return fail(WB_EINVAL, "B < 0");
  if (B == 0) return WB_OK;
  if (B > (int64_t)1 << 40) return fail(WB_EINVAL, "B too large");
  if (robot->dev.mimic_shared)
    return fail(WB_EINVAL, "the fused cost needs one link per joint (no shared mimic joints)");
  int rc;
  if ((rc = check_ptr(robot, q, "q", true))) return rc;
  if ((rc = check_ptr(robot, qd, "qd", true))) return rc;
  if ((rc = check_ptr(robot, qdd, "qdd", true))) return rc;
  if ((rc = check_ptr(robot, tau, "tau", true))) return rc;
  if ((rc = check_ptr(robot, tau_lo, "tau_lo", true))) return rc;
  if ((rc = check_ptr(robot, tau_hi, "tau_hi", true))) return rc;
  if ((rc = check_ptr(robot, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(robot, worst_pair, "worst_pair", d_min != nullptr))) return rc;
  if ((rc = check_ptr(robot, g_pose, "g_pose", false))) return rc;
  if ((rc = check_ptr(robot, g_sphere, "g_sphere", false))) return rc;
  if ((rc = check_ptr(robot, cost, "cost", false))) return rc;
  if ((rc = check_ptr(robot, gq, "gq", true))) return rc;
  if ((rc = check_ptr(robot, gqd, "gqd", true))) return rc;
  if ((rc = check_ptr(robot, gqdd, "gqdd", true))) return rc;
  if ((rc = check_ptr(robot, worst_diff, "worst_diff", false))) return rc;
  int kernel = tune ? tune->kernel : WB_KERNEL_AUTO;
  if (kernel == WB_KERNEL_TREE_NOCULL) kernel = WB_KERNEL_TREE;
  if (kernel != WB_KERNEL_AUTO && kernel != WB_KERNEL_TREE)
    return fail(WB_EINVAL, "the fused cost runs in the tree kernels (kernel AUTO or TREE)");
  if (robot->dev.maxdepth > tree_max_depth())
    return fail(WB_ETOOBIG, "tree deeper than %d levels", tree_max_depth());
  DeviceGuard guard(robot->device);
  BwdArgs a{B, q, qd, qdd, worst_pair, g_pose, g_sphere, nullptr, nullptr, gq, gqd, gqdd};
  a.wdiff = worst_diff;
  FusedCost fc;
  fc.tau = tau;
  fc.d_min = d_min;
  fc.lo = tau_lo;
  fc.hi = tau_hi;
  fc.w = W.collision;
  fc.smooth = W.smooth;
  fc.length = W.length;
  fc.e = W.energy * W.dt * W.dt;
  fc.cost = cost;
  const int tpb = (tune && tune->configs_per_block) ? tune->configs_per_block : 128;
  if (tpb < 32 || tpb > 512 || tpb % 32)
    return fail(WB_EINVAL, "tree threads per block must be a multiple of 32 in [32, 512]");
  int G = 1;
  if ((rc = tree_segments(robot, tune, B, tpb, false, &G))) return rc;
  const cudaError_t e =
      launch_tree_bwd(robot->dev, a, tpb, G, static_cast<cudaStream_t>(stream), &fc);
  if (e != cudaSuccess) return cuda_fail(e, "wb_eval_backward_cost launch");
  return WB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// uneven batches
// ---------------------------------------------------------------------------
struct wb_batch {
  int device = 0;
  int num_sms = 0;
  std::vector<wb_robot*> robots;
  std::vector<BatchProblemDev> probs;
  void* dmem = nullptr;
  const DevRobot* d_robots = nullptr;
  const PairSchedule32* d_scheds = nullptr;
  const BatchProblemDev* d_probs = nullptr;
  int4* d_titems[2] = {nullptr, nullptr};  // sweep items of the forward, backward pass
  const int2* d_pitems = nullptr;
  const int* d_counters = nullptr;
  int n_titems[2] = {0, 0};
  int cap_titems = 0;  // capacity of each sweep item list
  int n_pitems = 0;
  int ws_words = 0, rad_words = 0;
  int ns_max = 0;  // most shared slots among the used robots' 2-segment sweep plans
  wb_batch_sizes sizes{};
  // launch choices (wb_batch_set_tune / wb_batch_autotune): threads per block
  // of the forward and backward sweep passes, warps per block of the pair
  // pass (0 = the most that fit) and, per robot and pass, the sweep segments
  int threads[2] = {128, 128};
  int pair_warps = 0;
  std::vector<int> seg[2];
};

// the most shared output slots among these robots' 2-segment sweep plans
static int seg2_slots(const DevRobot& D) { return (D.seg_ok & 1) ? D.seg_ns[0] : 0; }

// default sweep segments of a robot: its 2-segment plan where it has one
static int default_segments(const DevRobot& D) { return (D.seg_ok & 1) ? 2 : 1; }

// Sweep items of a batch for per-robot segments (1 or 2), longest first: two
// segments sweep items of up to 32 configurations (mode 0), one segment
// items of up to 64 (mode 1, a warp each for 32); a robot without a
// 2-segment plan swept in mode 0 leaves the pair's second warp idle, so it
// always takes mode 1.
static std::vector<int4> batch_sweep_items(const wb_batch* Bt, const std::vector<int>& seg) {
  std::vector<int4> items;
  std::vector<int> cost;
  for (size_t p = 0; p < Bt->probs.size(); ++p) {
    const int ri = Bt->probs[p].robot, H = Bt->probs[p].H;
    const DevRobot& D = Bt->robots[ri]->dev;
    const bool two = seg[ri] == 2 && (D.seg_ok & 1);
    const int per = two ? 32 : 64;
    for (int c = 0; c < H; c += per) {
      items.push_back(make_int4((int)p, c, std::min(per, H - c), two ? 0 : 1));
      // links a warp walks: half the tree plus the replayed ancestors, or all
      cost.push_back(two ? (D.n + 1) / 2 + D.maxdepth / 2 : D.n);
    }
  }
  std::vector<int> order(items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int4> out;
  for (int i : order) out.push_back(items[i]);
  return out;
}

// upload the sweep items of pass (0 forward, 1 backward) for the batch's
// current segments (a setup-time copy)
static int batch_upload_items(wb_batch* Bt, int pass) {
  std::vector<int4> it = batch_sweep_items(Bt, Bt->seg[pass]);
  if ((int)it.size() > Bt->cap_titems) return fail(WB_ECUDA, "sweep items exceed capacity");
  Bt->n_titems[pass] = Bt->sizes.configs > 0 ? (int)it.size() : 0;
  if (it.empty()) return WB_OK;
  DeviceGuard guard(Bt->device);
  cudaError_t e =
      cudaMemcpy(Bt->d_titems[pass], it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? WB_OK : cuda_fail(e, "batch item upload");
}

extern "C" {

int wb_batch_create(wb_robot* const* robots, int32_t n_robots, const wb_problem* problems,
                    int32_t n_problems, wb_batch** out) {
  g_err.clear();
  if (!out) return fail(WB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!robots || n_robots <= 0) return fail(WB_EINVAL, "no robots");
  if (n_problems < 0 || (n_problems > 0 && !problems)) return fail(WB_EINVAL, "bad problems");
  const int dev = robots[0] ? robots[0]->device : -1;
  for (int i = 0; i < n_robots; ++i) {
    if (!robots[i]) return fail(WB_EINVAL, "robot %d is NULL", i);
    if (robots[i]->device != dev) return fail(WB_EDEVICE, "robots on different devices");
    if (robots[i]->dev.maxdepth > tree_max_depth())
      return fail(WB_ETOOBIG, "robot %d deeper than %d levels", i, tree_max_depth());
  }
  wb_batch* Bt = new wb_batch();
  Bt->device = dev;
  Bt->num_sms = robots[0]->num_sms;
  Bt->robots.assign(robots, robots + n_robots);
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < n_robots; ++i) Bt->seg[pass].push_back(default_segments(robots[i]->dev));
  int64_t jo = 0, po = 0, so = 0, co = 0;
  std::vector<int2> pitems;
  for (int p = 0; p < n_problems; ++p) {
    const int ri = problems[p].robot, H = problems[p].horizon;
    if (ri < 0 || ri >= n_robots) {
      delete Bt;
      return fail(WB_ERANGE, "problem %d: robot %d out of range", p, ri);
    }
    if (H < 0) {
      delete Bt;
      return fail(WB_EINVAL, "problem %d: horizon %d < 0", p, H);
    }
    const DevRobot& D = robots[ri]->dev;
    Bt->probs.push_back(BatchProblemDev{ri, H, jo, po, so, co});
    jo += (int64_t)D.d * H;
    po += (int64_t)H * D.n * 12;
    so += (int64_t)H * D.S * 3;
    co += H;
    Bt->cap_titems += (H + 31) / 32;
    for (int c = 0; c < H; ++c) pitems.push_back(make_int2(p, c));
    Bt->ws_words = std::max(Bt->ws_words, pair_plan_words(D));
    Bt->rad_words = std::max(Bt->rad_words, (4 * D.Sg + 31) & ~31);
    Bt->ns_max = std::max(Bt->ns_max, seg2_slots(D));
  }
  Bt->sizes = wb_batch_sizes{jo, po, so, co, n_problems, n_robots};
  // longest work first
  auto pcost = [&](const int2& w) { return robots[Bt->probs[w.x].robot]->dev.P; };
  std::stable_sort(pitems.begin(), pitems.end(),
                   [&](const int2& a, const int2& b) { return pcost(a) > pcost(b); });
  std::vector<DevRobot> drs;
  std::vector<PairSchedule32> dss;
  for (int i = 0; i < n_robots; ++i) {
    drs.push_back(robots[i]->dev);
    dss.push_back(robots[i]->sched32);
  }
  std::vector<int> counters(4, 0);
  std::vector<int4> titems(std::max(Bt->cap_titems, 1), make_int4(0, 0, 0, 0));
  if (pitems.empty()) pitems.push_back(make_int2(0, 0));
  std::vector<BatchProblemDev> probs_dev = Bt->probs;
  if (probs_dev.empty()) probs_dev.push_back(BatchProblemDev{0, 0, 0, 0, 0, 0});
  Bt->n_pitems = co > 0 ? (int)pitems.size() : 0;
  const int4* tslot[2] = {nullptr, nullptr};
  Packer pk;
  pk.add_vec(drs, &Bt->d_robots);
  pk.add_vec(dss, &Bt->d_scheds);
  pk.add_vec(probs_dev, &Bt->d_probs);
  pk.add_vec(titems, &tslot[0]);
  pk.add_vec(titems, &tslot[1]);
  pk.add_vec(pitems, &Bt->d_pitems);
  pk.add_vec(counters, &Bt->d_counters);
  DeviceGuard guard(dev);
  cudaError_t e = cudaMalloc(&Bt->dmem, pk.host.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(Bt->dmem, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (Bt->dmem) cudaFree(Bt->dmem);
    delete Bt;
    return cuda_fail(e, "batch upload");
  }
  for (auto& it : pk.items) *it.slot = static_cast<char*>(Bt->dmem) + it.off;
  Bt->d_titems[0] = const_cast<int4*>(tslot[0]);
  Bt->d_titems[1] = const_cast<int4*>(tslot[1]);
  for (int pass = 0; pass < 2; ++pass) {
    const int rc = batch_upload_items(Bt, pass);
    if (rc) {
      wb_free_batch(Bt);
      return rc;
    }
  }
  *out = Bt;
  return WB_OK;
}

int wb_batch_sizes_get(const wb_batch* batch, wb_batch_sizes* out) {
  if (!batch || !out) return fail(WB_EINVAL, "NULL argument");
  *out = batch->sizes;
  return WB_OK;
}

int wb_batch_offsets(const wb_batch* batch, int64_t* joint, int64_t* pose, int64_t* sphere,
                     int64_t* config) {
  if (!batch) return fail(WB_EINVAL, "batch is NULL");
  for (size_t p = 0; p < batch->probs.size(); ++p) {
    if (joint) joint[p] = batch->probs[p].jo;
    if (pose) pose[p] = batch->probs[p].po;
    if (sphere) sphere[p] = batch->probs[p].so;
    if (config) config[p] = batch->probs[p].co;
  }
  return WB_OK;
}

void wb_free_batch(wb_batch* batch) {
  if (!batch) return;
  {
    DeviceGuard guard(batch->device);
    if (batch->dmem) cudaFree(batch->dmem);
  }
  delete batch;
}

static int batch_grid_tree(const wb_batch* Bt, bool fwd, int* grid) {
  const int pass = fwd ? 0 : 1, threads = Bt->threads[pass];
  int bps = 0;
  cudaError_t e = batch_tree_max_blocks_per_sm(fwd, Bt->ns_max, threads, &bps);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(WB_ETOOBIG, "batch sweep block of %d threads does not fit", threads);
  const int pairs = threads / 64;  // an item per pair of warps
  const int need = (Bt->n_titems[pass] + pairs - 1) / pairs;
  *grid = std::max(1, std::min(need, bps * Bt->num_sms));
  return WB_OK;
}

// the pair pass's warps per block: the batch's choice, or the most that fit
static int batch_pair_warps(const wb_batch* Bt) {
  const int most = warps_that_fit(0, batch_pair_smem(Bt->ws_words, Bt->rad_words, 1));
  return Bt->pair_warps > 0 ? std::min(Bt->pair_warps, most) : most;
}

int wb_batch_eval(wb_batch* batch, const float* q, const float* qd, const float* qdd,
                  float* link_pose, float* sphere, float* d_min, int32_t* worst_pair, float* tau,
                  void* stream) {
  g_err.clear();
  if (!batch) return fail(WB_EINVAL, "batch is NULL");
  if (batch->sizes.configs == 0) return WB_OK;
  const wb_robot* R0 = batch->robots[0];
  int rc;
  if ((rc = check_ptr(R0, q, "q", true))) return rc;
  if ((rc = check_ptr(R0, qd, "qd", tau != nullptr))) return rc;
  if ((rc = check_ptr(R0, qdd, "qdd", tau != nullptr))) return rc;
  const bool pairs = d_min || sphere;
  if ((rc = check_ptr(R0, link_pose, "link_pose", pairs))) return rc;
  if ((rc = check_ptr(R0, sphere, "sphere", false))) return rc;
  if ((rc = check_ptr(R0, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(R0, worst_pair, "worst_pair", d_min != nullptr))) return rc;
  if ((rc = check_ptr(R0, tau, "tau", false))) return rc;
  if (!d_min && worst_pair) return fail(WB_EINVAL, "worst_pair without d_min");
  DeviceGuard guard(batch->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BatchIO io{q, qd, qdd, link_pose, sphere, d_min, worst_pair, tau,
             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int* counters = const_cast<int*>(batch->d_counters);
  cudaError_t e = cudaSuccess;
  if (link_pose || tau) {
    int grid = 1;
    if ((rc = batch_grid_tree(batch, true, &grid))) return rc;
    e = launch_batch_tree_fwd(batch->d_robots, batch->d_probs, batch->d_titems[0],
                              batch->n_titems[0], counters, io, grid, batch->ns_max,
                              batch->threads[0], s);
    if (e != cudaSuccess) return cuda_fail(e, "wb_batch_eval launch");
  }
  if (pairs && batch->n_pitems > 0) {
    const int warps = batch_pair_warps(batch);
    if (warps == 0) return fail(WB_ETOOBIG, "batch pair kernel does not fit on an SM");
    int bps = 0;
    e = batch_pair_max_blocks_per_sm(warps, batch->ws_words, batch->rad_words, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (bps < 1) return fail(WB_ETOOBIG, "batch pair kernel does not fit on an SM");
    const int need = (batch->n_pitems + warps - 1) / warps;
    const int grid = std::min(need, bps * batch->num_sms);
    e = launch_batch_pair(batch->d_robots, batch->d_scheds, batch->d_probs, batch->d_pitems,
                          batch->n_pitems, counters + 1, io, grid, warps, batch->ws_words,
                          batch->rad_words, s);
    if (e != cudaSuccess) return cuda_fail(e, "wb_batch_eval launch");
  }
  return WB_OK;
}

int wb_batch_eval_backward(wb_batch* batch, const float* q, const float* qd, const float* qdd,
                           const int32_t* worst_pair, const float* g_pose, const float* g_sphere,
                           const float* g_dmin, const float* g_tau, float* gq, float* gqd,
                           float* gqdd, void* stream) {
  g_err.clear();
  if (!batch) return fail(WB_EINVAL, "batch is NULL");
  if (batch->sizes.configs == 0) return WB_OK;
  const wb_robot* R0 = batch->robots[0];
  int rc;
  if ((rc = check_ptr(R0, q, "q", true))) return rc;
  if ((rc = check_ptr(R0, qd, "qd", true))) return rc;
  if ((rc = check_ptr(R0, qdd, "qdd", true))) return rc;
  if ((rc = check_ptr(R0, worst_pair, "worst_pair", g_dmin != nullptr))) return rc;
  if ((rc = check_ptr(R0, g_pose, "g_pose", false))) return rc;
  if ((rc = check_ptr(R0, g_sphere, "g_sphere", false))) return rc;
  if ((rc = check_ptr(R0, g_dmin, "g_dmin", false))) return rc;
  if ((rc = check_ptr(R0, g_tau, "g_tau", false))) return rc;
  if ((rc = check_ptr(R0, gq, "gq", true))) return rc;
  if ((rc = check_ptr(R0, gqd, "gqd", true))) return rc;
  if ((rc = check_ptr(R0, gqdd, "gqdd", true))) return rc;
  DeviceGuard guard(batch->device);
  BatchIO io{q, qd, qdd, nullptr, nullptr, nullptr, const_cast<int32_t*>(worst_pair), nullptr,
             g_pose, g_sphere, g_dmin, g_tau, gq, gqd, gqdd};
  int grid = 1;
  if ((rc = batch_grid_tree(batch, false, &grid))) return rc;
  cudaError_t e = launch_batch_tree_bwd(batch->d_robots, batch->d_probs, batch->d_titems[1],
                                        batch->n_titems[1], const_cast<int*>(batch->d_counters) + 2,
                                        io, grid, batch->ns_max, batch->threads[1],
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_batch_eval_backward launch");
  return WB_OK;
}

int wb_batch_set_tune(wb_batch* batch, const wb_batch_tune* tune, const int32_t* fwd_segments,
                      const int32_t* bwd_segments) {
  g_err.clear();
  if (!batch) return fail(WB_EINVAL, "batch is NULL");
  const int nr = (int)batch->robots.size();
  wb_batch_tune t = tune ? *tune : wb_batch_tune{0, 0, 0};
  for (int x : {t.fwd_threads, t.bwd_threads})
    if (x != 0 && x != 64 && x != 128 && x != 256)
      return fail(WB_EINVAL, "sweep threads per block %d: 0, 64, 128 or 256", x);
  if (t.pair_warps < 0 || t.pair_warps > 8)
    return fail(WB_EINVAL, "pair warps per block %d: 0..8", t.pair_warps);
  const int most = warps_that_fit(0, batch_pair_smem(batch->ws_words, batch->rad_words, 1));
  if (t.pair_warps > most)
    return fail(WB_ETOOBIG, "%d pair warps per block do not fit (at most %d)", t.pair_warps, most);
  const int32_t* segs[2] = {fwd_segments, bwd_segments};
  std::vector<int> next[2];
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < nr; ++i) {
      const DevRobot& D = batch->robots[i]->dev;
      const int g = segs[pass] ? segs[pass][i] : default_segments(D);
      if (g != 1 && g != 2) return fail(WB_EINVAL, "robot %d: %d segments (1 or 2)", i, g);
      if (g == 2 && !(D.seg_ok & 1))
        return fail(WB_EINVAL, "robot %d has no 2-segment sweep plan", i);
      next[pass].push_back(g);
    }
  batch->threads[0] = t.fwd_threads ? t.fwd_threads : 128;
  batch->threads[1] = t.bwd_threads ? t.bwd_threads : 128;
  batch->pair_warps = t.pair_warps;
  for (int pass = 0; pass < 2; ++pass) {
    batch->seg[pass] = next[pass];
    const int rc = batch_upload_items(batch, pass);
    if (rc) return rc;
  }
  return WB_OK;
}

int wb_batch_get_tune(const wb_batch* batch, wb_batch_tune* tune, int32_t* fwd_segments,
                      int32_t* bwd_segments) {
  if (!batch) return fail(WB_EINVAL, "batch is NULL");
  if (tune) *tune = wb_batch_tune{batch->threads[0], batch->threads[1], batch->pair_warps};
  for (size_t i = 0; i < batch->robots.size(); ++i) {
    if (fwd_segments) fwd_segments[i] = batch->seg[0][i];
    if (bwd_segments) bwd_segments[i] = batch->seg[1][i];
  }
  return WB_OK;
}

// ---------------------------------------------------------------------------
// trajectory-optimisation ends
// ---------------------------------------------------------------------------
// A device buffer of the call: NULL only when optional, 16-byte aligned,
// device memory; the first one fixes the call's device (-1 = not yet known).
static int check_buf(const void* p, const char* name, bool required, int* device) {
  if (!p) return required ? fail(WB_EINVAL, "%s is NULL", name) : WB_OK;
  if (reinterpret_cast<uintptr_t>(p) & 15u)
    return fail(WB_EINVAL, "%s is not 16-byte aligned", name);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(WB_EDEVICE, "%s: not a CUDA pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(WB_EDEVICE, "%s is not device memory", name);
  if (at.type == cudaMemoryTypeDevice) {
    if (*device < 0) *device = at.device;
    else if (at.device != *device)
      return fail(WB_EDEVICE, "%s lives on device %d, other buffers on device %d", name,
                  at.device, *device);
  }
  return WB_OK;
}

// K control points extended by 3 ghost knots (has_start) and 3 repeats of
// the last one (end_static) must give at least one cubic segment
static int check_spline(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                        int has_start = 0, int end_static = 0) {
  if (n_traj < 0 || d < 1 || d > WB_MAX_LINKS) return fail(WB_EINVAL, "bad n_traj or d");
  const int Kx = K + (has_start ? 3 : 0) + (end_static ? 3 : 0);
  if (K < 1 || K > 4096 || Kx < 4)
    return fail(WB_EINVAL,
                "K = %d outside [1, 4096] or fewer than 4 knots with the boundary conditions "
                "(a cubic B-spline needs 4)", K);
  if (T < 2 || T > 4096) return fail(WB_EINVAL, "T = %d outside [2, 4096]", T);
  if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(WB_EINVAL, "dt must be positive");
  if (n_traj * T * (int64_t)d > ((int64_t)1 << 40)) return fail(WB_EINVAL, "too many samples");
  return WB_OK;
}

int wb_bspline_eval_bc(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt, const float* U,
                       const float* start, int32_t end_static, float* q, float* qd, float* qdd,
                       void* stream) {
  g_err.clear();
  int rc, dev = -1;
  if ((rc = check_spline(n_traj, d, K, T, dt, start != nullptr, end_static))) return rc;
  if ((rc = check_buf(U, "U", n_traj > 0, &dev))) return rc;
  if ((rc = check_buf(start, "start", false, &dev))) return rc;
  if ((rc = check_buf(q, "q", false, &dev))) return rc;
  if ((rc = check_buf(qd, "qd", false, &dev))) return rc;
  if ((rc = check_buf(qdd, "qdd", false, &dev))) return rc;
  if (n_traj == 0 || (!q && !qd && !qdd)) return WB_OK;
  DeviceGuard guard(dev);
  cudaError_t e = launch_bspline_fwd(n_traj, d, K, T, dt, U, start, end_static, q, qd, qdd,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_bspline_eval launch");
  return WB_OK;
}

int wb_bspline_eval(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt, const float* U,
                    float* q, float* qd, float* qdd, void* stream) {
  if (K < 4) {
    g_err.clear();
    return fail(WB_EINVAL, "K = %d outside [4, 4096] (a cubic B-spline needs 4 control points)",
                K);
  }
  return wb_bspline_eval_bc(n_traj, d, K, T, dt, U, nullptr, 0, q, qd, qdd, stream);
}

int wb_bspline_backward_bc(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                           int32_t has_start, int32_t end_static, const float* gq,
                           const float* gqd, const float* gqdd, const float* gqd_add,
                           const float* gqdd_add, float* gU, float* g_start, void* stream) {
  g_err.clear();
  int rc, dev = -1;
  if ((rc = check_spline(n_traj, d, K, T, dt, has_start, end_static))) return rc;
  if (g_start && !has_start) return fail(WB_EINVAL, "g_start without has_start");
  if ((rc = check_buf(gU, "gU", n_traj > 0, &dev))) return rc;
  if ((rc = check_buf(g_start, "g_start", false, &dev))) return rc;
  if ((rc = check_buf(gq, "gq", false, &dev))) return rc;
  if ((rc = check_buf(gqd, "gqd", false, &dev))) return rc;
  if ((rc = check_buf(gqdd, "gqdd", false, &dev))) return rc;
  if ((rc = check_buf(gqd_add, "gqd_add", false, &dev))) return rc;
  if ((rc = check_buf(gqdd_add, "gqdd_add", false, &dev))) return rc;
  if (n_traj == 0) return WB_OK;
  DeviceGuard guard(dev);
  cudaError_t e = launch_bspline_bwd(n_traj, d, K, T, dt, has_start, end_static, gq, gqd, gqdd,
                                     gqd_add, gqdd_add, gU, g_start,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_bspline_backward launch");
  return WB_OK;
}

int wb_bspline_backward_ext(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                            const float* gq, const float* gqd, const float* gqdd,
                            const float* gqd_add, const float* gqdd_add, float* gU,
                            void* stream) {
  if (K < 4) {
    g_err.clear();
    return fail(WB_EINVAL, "K = %d outside [4, 4096] (a cubic B-spline needs 4 control points)",
                K);
  }
  return wb_bspline_backward_bc(n_traj, d, K, T, dt, 0, 0, gq, gqd, gqdd, gqd_add, gqdd_add, gU,
                                nullptr, stream);
}

int wb_bspline_backward(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                        const float* gq, const float* gqd, const float* gqdd, float* gU,
                        void* stream) {
  return wb_bspline_backward_ext(n_traj, d, K, T, dt, gq, gqd, gqdd, nullptr, nullptr, gU,
                                 stream);
}

int wb_trajopt_cost_ext(int64_t B, int32_t d, const float* tau, const float* d_min,
                        const float* qd, const float* qdd, const float* tau_lo,
                        const float* tau_hi, const wb_cost_weights* w, float* cost,
                        float* g_tau, float* g_dmin, float* g_qd, float* g_qdd, void* stream) {
  g_err.clear();
  int rc, dev = -1;
  if (!w) return fail(WB_EINVAL, "weights are NULL");
  const wb_cost_weights W = *w;
  if (B < 0 || d < 0 || d > WB_MAX_LINKS) return fail(WB_EINVAL, "bad B or d");
  if (B * (int64_t)std::max(d, 1) > ((int64_t)1 << 40)) return fail(WB_EINVAL, "B too large");
  if (!std::isfinite(W.collision) || !std::isfinite(W.smooth) || !std::isfinite(W.length) ||
      !std::isfinite(W.energy) || !std::isfinite(W.dt) || !(W.dt > 0.0f) ||
      !std::isfinite(W.energy * W.dt * W.dt))
    return fail(WB_EINVAL, "weights must be finite and dt > 0");
  if ((rc = check_buf(tau, "tau", false, &dev))) return rc;
  if ((rc = check_buf(d_min, "d_min", false, &dev))) return rc;
  if ((rc = check_buf(qd, "qd", false, &dev))) return rc;
  if ((rc = check_buf(qdd, "qdd", false, &dev))) return rc;
  if ((rc = check_buf(tau_lo, "tau_lo", tau != nullptr, &dev))) return rc;
  if ((rc = check_buf(tau_hi, "tau_hi", tau != nullptr, &dev))) return rc;
  if ((rc = check_buf(cost, "cost", false, &dev))) return rc;
  if ((rc = check_buf(g_tau, "g_tau", false, &dev))) return rc;
  if ((rc = check_buf(g_dmin, "g_dmin", false, &dev))) return rc;
  if ((rc = check_buf(g_qd, "g_qd", false, &dev))) return rc;
  if ((rc = check_buf(g_qdd, "g_qdd", false, &dev))) return rc;
  if (g_tau && !tau) return fail(WB_EINVAL, "g_tau without tau");
  if (g_dmin && !d_min) return fail(WB_EINVAL, "g_dmin without d_min");
  if (B == 0 || dev < 0) return WB_OK;
  DeviceGuard guard(dev);
  cudaError_t e = launch_trajopt_cost(B, d, tau, d_min, qd, qdd, tau_lo, tau_hi, W.collision,
                                      W.smooth, W.length, W.energy * W.dt * W.dt, cost, g_tau,
                                      g_dmin, g_qd, g_qdd, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wb_trajopt_cost launch");
  return WB_OK;
}

int wb_trajopt_cost(int64_t B, int32_t d, const float* tau, const float* d_min,
                    const float* tau_lo, const float* tau_hi, float w_coll, float* cost,
                    float* g_tau, float* g_dmin, void* stream) {
  const wb_cost_weights w = {w_coll, 0.0f, 0.0f, 0.0f, 1.0f};
  return wb_trajopt_cost_ext(B, d, tau, d_min, nullptr, nullptr, tau_lo, tau_hi, &w, cost, g_tau,
                             g_dmin, nullptr, nullptr, stream);
}

// The work tables of wb_batch_create, rebuilt per call in the library's static
// scratch (k_noalloc.cu) instead of device memory allocated per batch.  The
// host fills the setup kernel's launch parameters (NoAllocPlan, on this
// stack) and chooses the same longest-first order of work items.
int wb_batch_eval_noalloc(wb_robot* const* robots, int32_t n_robots, const wb_problem* problems,
                          int32_t n_problems, const float* q, const float* qd, const float* qdd,
                          float* link_pose, float* sphere, float* d_min, int32_t* worst_pair,
                          float* tau, void* stream) {
  g_err.clear();
  if (!robots || n_robots <= 0) return fail(WB_EINVAL, "no robots");
  if (n_problems < 0 || (n_problems > 0 && !problems)) return fail(WB_EINVAL, "bad problems");
  if (n_robots > WB_NOALLOC_MAX_ROBOTS)
    return fail(WB_ETOOBIG, "%d robots: at most %d per call", n_robots, WB_NOALLOC_MAX_ROBOTS);
  if (n_problems > WB_NOALLOC_MAX_PROBLEMS)
    return fail(WB_ETOOBIG, "%d problems: at most %d per call", n_problems,
                WB_NOALLOC_MAX_PROBLEMS);
  static_assert(WB_NOALLOC_MAX_ROBOTS == NA_MAX_ROBOTS &&
                    WB_NOALLOC_MAX_PROBLEMS == NA_MAX_PROBLEMS &&
                    WB_NOALLOC_MAX_CONFIGS == NA_MAX_CONFIGS,
                "public and internal limits differ");
  const int dev = robots[0] ? robots[0]->device : -1;
  for (int i = 0; i < n_robots; ++i) {
    if (!robots[i]) return fail(WB_EINVAL, "robot %d is NULL", i);
    if (robots[i]->device != dev) return fail(WB_EDEVICE, "robots on different devices");
    if (robots[i]->dev.maxdepth > tree_max_depth())
      return fail(WB_ETOOBIG, "robot %d deeper than %d levels", i, tree_max_depth());
  }
  int64_t configs = 0;
  for (int p = 0; p < n_problems; ++p) {
    const int ri = problems[p].robot, H = problems[p].horizon;
    if (ri < 0 || ri >= n_robots) return fail(WB_ERANGE, "problem %d: robot %d out of range", p, ri);
    if (H < 0) return fail(WB_EINVAL, "problem %d: horizon %d < 0", p, H);
    configs += H;
    if (configs > WB_NOALLOC_MAX_CONFIGS)
      return fail(WB_ETOOBIG, "more than %d configurations per call", WB_NOALLOC_MAX_CONFIGS);
  }
  const wb_robot* R0 = robots[0];
  int rc;
  if ((rc = check_ptr(R0, q, "q", configs > 0))) return rc;
  if ((rc = check_ptr(R0, qd, "qd", configs > 0 && tau != nullptr))) return rc;
  if ((rc = check_ptr(R0, qdd, "qdd", configs > 0 && tau != nullptr))) return rc;
  const bool pairs = d_min || sphere;
  if ((rc = check_ptr(R0, link_pose, "link_pose", configs > 0 && pairs))) return rc;
  if ((rc = check_ptr(R0, sphere, "sphere", false))) return rc;
  if ((rc = check_ptr(R0, d_min, "d_min", false))) return rc;
  if ((rc = check_ptr(R0, worst_pair, "worst_pair", configs > 0 && d_min != nullptr))) return rc;
  if ((rc = check_ptr(R0, tau, "tau", false))) return rc;
  if (!d_min && worst_pair) return fail(WB_EINVAL, "worst_pair without d_min");
  if (configs == 0) return WB_OK;

  NoAllocPlan plan;
  plan.n_robots = n_robots;
  plan.n_problems = n_problems;
  plan.n_configs = (int)configs;
  int ws_words = 0, rad_words = 0, ns_max = 0;
  for (int i = 0; i < n_robots; ++i) {
    plan.robots[i] = robots[i]->dev;
    plan.scheds[i] = robots[i]->sched32;
  }
  // shared-memory sizes over the robots that some problem uses, as
  // wb_batch_create takes them
  for (int p = 0; p < n_problems; ++p) {
    const DevRobot& D = robots[problems[p].robot]->dev;
    plan.prob[p] = problems[p].robot << 24 | problems[p].horizon;
    ws_words = std::max(ws_words, pair_plan_words(D));
    rad_words = std::max(rad_words, (4 * D.Sg + 31) & ~31);
    ns_max = std::max(ns_max, seg2_slots(D));
  }
  // longest work first: robots by cost (stable), problems in order within one
  int n_titems = 0, n_pitems = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int order[NA_MAX_ROBOTS];
    for (int i = 0; i < n_robots; ++i) order[i] = i;
    auto cost = [&](int i) { return pass == 0 ? robots[i]->dev.n : robots[i]->dev.P; };
    std::stable_sort(order, order + n_robots, [&](int a, int b) { return cost(a) > cost(b); });
    int next = 0;
    for (int k = 0; k < n_robots; ++k)
      for (int p = 0; p < n_problems; ++p) {
        if (problems[p].robot != order[k]) continue;
        const int H = problems[p].horizon;
        if (pass == 0) {
          plan.tstart[p] = next;
          next += (H + 31) / 32;
        } else {
          plan.pstart[p] = next;
          next += H;
        }
      }
    (pass == 0 ? n_titems : n_pitems) = next;
  }

  DeviceGuard guard(dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  cudaError_t e = noalloc_scratch(dev, &base);
  if (e != cudaSuccess) return cuda_fail(e, "scratch address lookup");
  const NoAllocTables T = noalloc_tables(base);
  const int setup_grid = std::max(1, std::min((n_pitems + 1023) / 1024, R0->num_sms));
  e = launch_noalloc_setup(plan, base, setup_grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "wb_batch_eval_noalloc setup launch");
  BatchIO io{q, qd, qdd, link_pose, sphere, d_min, worst_pair, tau,
             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (link_pose || tau) {
    int bps = 0;
    e = batch_tree_max_blocks_per_sm(true, ns_max, 128, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    const int grid = std::max(1, std::min((n_titems + 1) / 2, std::max(bps, 1) * R0->num_sms));
    e = launch_batch_tree_fwd(T.robots, T.probs, T.titems, n_titems, T.counters, io, grid, ns_max,
                              128, s);
    if (e != cudaSuccess) return cuda_fail(e, "wb_batch_eval_noalloc launch");
  }
  if (pairs) {
    const int warps = warps_that_fit(0, batch_pair_smem(ws_words, rad_words, 1));
    if (warps == 0) return fail(WB_ETOOBIG, "batch pair kernel does not fit on an SM");
    int bps = 0;
    e = batch_pair_max_blocks_per_sm(warps, ws_words, rad_words, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (bps < 1) return fail(WB_ETOOBIG, "batch pair kernel does not fit on an SM");
    const int grid = std::min((n_pitems + warps - 1) / warps, bps * R0->num_sms);
    e = launch_batch_pair(T.robots, T.scheds, T.probs, T.pitems, n_pitems, T.counters + 1, io, grid,
                          warps, ws_words, rad_words, s);
    if (e != cudaSuccess) return cuda_fail(e, "wb_batch_eval_noalloc launch");
  }
  return WB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {
struct Scratch {
  std::vector<void*> bufs;
  ~Scratch() {
    for (void* p : bufs) cudaFree(p);
  }
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return static_cast<T*>(p);
  }
};

float median_of(std::vector<float> v) {
  std::sort(v.begin(), v.end());
  return v[v.size() / 2];
}

// The autotuners' clock: the median of kTuneReps runs of f on stream s, each
// after an L2 flush (a memset of flush_bytes, outside the events), as a step
// over a batch that does not stay in L2 sees it.  pre() runs between the
// flush and the timed region: a backward candidate is timed after the
// forward sweep and the pair stage that precede it in a step, so that it
// finds the cache as it does there (timed straight after the flush, the
// control-point backward's 2 x 512 and 1 x 256 shapes ranked within 1 % of
// each other and the choice flipped between runs, where the trajectory step
// runs them at 0.127 and 0.132 ms).
constexpr int kTuneReps = 5;
struct TuneClock {
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* flush = nullptr;
  size_t flush_bytes = 0;
  bool init(Scratch& sc, int device) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return false;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) == cudaSuccess && l2 > 0) {
      flush_bytes = 2 * (size_t)l2;
      flush = sc.get<char>(flush_bytes);  // no flush if it cannot be had
      if (!flush) cudaGetLastError();
    }
    return true;
  }
  template <class F, class P>
  float time(F&& f, P&& pre) {
    std::vector<float> ts;
    for (int rep = 0; rep < kTuneReps; ++rep) {
      if (flush) cudaMemsetAsync(flush, rep & 0xFF, flush_bytes, s);
      pre();
      cudaEventRecord(e0, s);
      f();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ts.push_back(ms);
    }
    return median_of(ts);
  }
  template <class F>
  float time(F&& f) {
    return time(f, [] {});
  }
  ~TuneClock() {
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
  }
};

// the depth-first sweep shapes a robot takes for B configurations: segments
// x threads per block -- 64 / 128 / 256, 512 for the segmented sweeps (one
// block per SM then holds the link parameters once), and the balanced block
// that deals the batch's 32-configuration groups evenly over the SMs in one
// wave (448 threads at 2 segments for 32768 configurations on 152 SMs: 147
// blocks of 14 warps, where 512-thread blocks leave 24 SMs idle)
std::vector<wb_tune> sweep_shapes(const DevRobot& D, bool pair_warps, int64_t B, int num_sms) {
  std::vector<wb_tune> c;
  if (D.maxdepth > tree_max_depth()) return c;
  const int64_t groups = (B + 31) / 32;
  for (int seg : {1, 2, 4, 8}) {
    const bool ok = seg == 1 || (D.seg_ok >> (seg == 2 ? 0 : seg == 4 ? 1 : 2) & 1);
    if (!ok) continue;
    const int lim = seg == 1 ? 256 : 512;
    const int64_t per_sm = num_sms > 0 ? (seg == 1 ? (B + num_sms - 1) / num_sms
                                                   : (groups + num_sms - 1) / num_sms)
                                       : 0;
    const int64_t bal = seg == 1 ? (per_sm + 31) / 32 * 32 : 32 * seg * per_sm;
    std::vector<int> tpbs = {64, 128, 256, 512};
    if (bal >= 32 && bal <= lim && bal != 64 && bal != 128 && bal != 256 && bal != 512)
      tpbs.push_back((int)bal);
    for (int tpb : tpbs) {
      if (tpb > lim || (seg > 1 && tpb < 128)) continue;
      for (int pw : {4, 8}) {
        if (!pair_warps && pw == 8) continue;
        c.push_back(wb_tune{WB_KERNEL_TREE, seg, tpb, pair_warps ? pw : 0});
      }
    }
  }
  return c;
}
}  // namespace

extern "C" int wb_autotune(wb_robot* robot, int64_t B, wb_tune* fwd, wb_tune* bwd, float* fwd_ms,
                           float* bwd_ms) {
  g_err.clear();
  if (!robot || !fwd || !bwd) return fail(WB_EINVAL, "NULL argument");
  if (B <= 0) return fail(WB_EINVAL, "B must be positive");
  DeviceGuard guard(robot->device);
  const DevRobot& D = robot->dev;
  Scratch sc;
  const size_t nj = (size_t)D.d * B;
  float* q = sc.get<float>(nj);
  float* qd = sc.get<float>(nj);
  float* qdd = sc.get<float>(nj);
  float* pose = sc.get<float>((size_t)B * D.n * 12);
  float* sph = sc.get<float>((size_t)B * D.S * 3);
  float* dmin = sc.get<float>(B);
  int32_t* worst = sc.get<int32_t>(B);
  float* tau = sc.get<float>(nj);
  float* gpose = sc.get<float>((size_t)B * D.n * 12);
  float* gsph = sc.get<float>((size_t)B * D.S * 3);
  float* gdmin = sc.get<float>(B);
  float* gtau = sc.get<float>(nj);
  float* gq = sc.get<float>(nj);
  float* gqd = sc.get<float>(nj);
  float* gqdd = sc.get<float>(nj);
  if (!gqdd || !q || !pose || !sph || !gpose || !gsph) return fail(WB_ECUDA, "autotune scratch");
  {  // deterministic states: q in [-pi, pi], rates in [-2, 2], grads in [-1, 1]
    std::vector<float> h(std::max(nj, (size_t)B * std::max(D.n * 12, D.S * 3)));
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto uni = [&]() {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      return (float)((st >> 40) * (1.0 / 16777216.0)) * 2.0f - 1.0f;
    };
    auto fill = [&](float* dst, size_t n, float scale) {
      for (size_t i = 0; i < n; ++i) h[i] = scale * uni();
      return cudaMemcpy(dst, h.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    };
    cudaError_t e = fill(q, nj, 3.14159265f);
    if (e == cudaSuccess) e = fill(qd, nj, 2.0f);
    if (e == cudaSuccess) e = fill(qdd, nj, 5.0f);
    if (e == cudaSuccess) e = fill(gpose, (size_t)B * D.n * 12, 1.0f);
    if (e == cudaSuccess) e = fill(gsph, (size_t)B * D.S * 3, 1.0f);
    if (e == cudaSuccess) e = fill(gdmin, B, 1.0f);
    if (e == cudaSuccess) e = fill(gtau, nj, 1.0f);
    if (e != cudaSuccess) return cuda_fail(e, "autotune inputs");
  }
  TuneClock clk;
  if (!clk.init(sc, robot->device)) return fail(WB_ECUDA, "autotune stream/events");
  cudaStream_t s = clk.s;
  // the worst pairs and their centre differences the backward candidates
  // read, from the split forward (sweep, then the pair stage) as a step hands
  // them over; the forward candidates write their own worst pairs
  int32_t* worst_f = sc.get<int32_t>(B);
  float* dmin_f = sc.get<float>(B);
  float* wdiff = sc.get<float>(3 * (size_t)B);
  if (!worst_f || !dmin_f || !wdiff) return fail(WB_ECUDA, "autotune scratch");
  bool have_diff = false;
  if (D.maxdepth <= tree_max_depth()) {
    const wb_tune tt{WB_KERNEL_TREE, 0, 0, 0};
    have_diff = wb_eval(robot, B, q, qd, qdd, pose, nullptr, nullptr, nullptr, nullptr,
                        nullptr, &tt, s) == WB_OK &&
                wb_self_collision_dir(robot, B, pose, nullptr, dmin, worst, wdiff, nullptr,
                                      nullptr, s) == WB_OK;
  }
  if (!have_diff) {  // the fused fallback: its own forward's worst pairs
    const int rc0 = wb_eval(robot, B, q, qd, qdd, pose, nullptr, dmin, worst, nullptr, nullptr,
                            nullptr, s);
    if (rc0 != WB_OK) return rc0;
  }
  std::vector<wb_tune> cands = sweep_shapes(D, true, B, robot->num_sms);
  for (int G : {4, 8, 16, 32}) cands.push_back(wb_tune{WB_KERNEL_FUSED, G, 0, 0});
  if (plain_fits(D)) cands.push_back(wb_tune{WB_KERNEL_PLAIN, 0, 0, 0});
  float best_f = 1e30f, best_b = 1e30f;
  wb_tune bf = cands[0], bb = cands[0];
  for (const wb_tune& t : cands) {
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1 && t.kernel == WB_KERNEL_TREE && t.blocks_per_sm != 8) continue;
      auto run = [&]() {
        return pass == 0 ? wb_eval(robot, B, q, qd, qdd, pose, sph, dmin_f, worst_f, tau,
                                   nullptr, &t, s)
                         : wb_eval_backward_dir(robot, B, q, qd, qdd, nullptr, worst,
                                                have_diff ? wdiff : nullptr, gpose, gsph, gdmin,
                                                gtau, gq, gqd, gqdd, nullptr, &t, s);
      };
      if (run() != WB_OK) continue;  // shape not applicable to this robot
      // a backward candidate after the forward sweep and pair stage of a step
      auto pre = [&]() {
        if (pass == 1)
          wb_eval(robot, B, q, qd, qdd, pose, sph, dmin_f, worst_f, tau, nullptr, nullptr, s);
      };
      const float m = clk.time(run, pre);
      if (pass == 0 && m < best_f) {
        best_f = m;
        bf = t;
      }
      if (pass == 1 && m < best_b) {
        best_b = m;
        bb = t;
      }
    }
  }
  cudaStreamSynchronize(s);
  g_err.clear();
  *fwd = bf;
  *bwd = bb;
  if (fwd_ms) *fwd_ms = best_f;
  if (bwd_ms) *bwd_ms = best_b;
  return WB_OK;
}

extern "C" int wb_autotune_spline(wb_robot* robot, int64_t n_traj, int32_t K, int32_t T, float dt,
                                  const wb_cost_weights* w, wb_tune* fwd, wb_tune* bwd,
                                  float* fwd_ms, float* bwd_ms) {
  g_err.clear();
  if (!robot || !fwd || !bwd || !w) return fail(WB_EINVAL, "NULL argument");
  if (n_traj <= 0 || K < 4 || K > 4096 || T < 2 || T > 4096 || !(dt > 0.0f))
    return fail(WB_EINVAL, "spline sizes out of range");
  DeviceGuard guard(robot->device);
  const DevRobot& D = robot->dev;
  const int64_t B = n_traj * T;
  std::vector<wb_tune> cands = sweep_shapes(D, false, B, robot->num_sms);
  if (cands.empty()) return fail(WB_ETOOBIG, "tree deeper than the sweep kernels take");
  const size_t nj = (size_t)D.d * B;
  Scratch sc;
  float* U = sc.get<float>((size_t)n_traj * D.d * K);
  float* pose = sc.get<float>((size_t)B * D.n * 12);
  float* sph = sc.get<float>((size_t)B * D.S * 3);
  float* dmin = sc.get<float>(B);
  int32_t* worst = sc.get<int32_t>(B);
  float* tau = sc.get<float>(nj);
  float* cost = sc.get<float>(B);
  float* gq = sc.get<float>(nj);
  float* gqd = sc.get<float>(nj);
  float* gqdd = sc.get<float>(nj);
  float* lim = sc.get<float>(2 * (size_t)D.d);
  if (!U || !pose || !sph || !dmin || !worst || !tau || !cost || !gq || !gqd || !gqdd || !lim)
    return fail(WB_ECUDA, "autotune scratch");
  {  // deterministic control points in [-pi/2, pi/2]; torque limits +-30
    const size_t nu = (size_t)n_traj * D.d * K;
    std::vector<float> h(std::max(nu, 2 * (size_t)D.d));
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (size_t i = 0; i < nu; ++i) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      h[i] = 1.57079633f * ((float)((st >> 40) * (1.0 / 16777216.0)) * 2.0f - 1.0f);
    }
    cudaError_t e = cudaMemcpy(U, h.data(), nu * sizeof(float), cudaMemcpyHostToDevice);
    for (int j = 0; j < D.d; ++j) {
      h[j] = -30.0f;
      h[D.d + j] = 30.0f;
    }
    if (e == cudaSuccess)
      e = cudaMemcpy(lim, h.data(), 2 * (size_t)D.d * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "autotune inputs");
  }
  TuneClock clk;
  if (!clk.init(sc, robot->device)) return fail(WB_ECUDA, "autotune stream/events");
  cudaStream_t s = clk.s;
  const wb_spline sp{U, n_traj, K, T, dt};
  // the worst pairs, their centre differences and the torques the backward
  // reads, as the split forward (sweep, then the pair stage) hands them over
  float* wdiff = sc.get<float>(3 * (size_t)B);
  if (!wdiff) return fail(WB_ECUDA, "autotune scratch");
  int rc = wb_eval_spline(robot, &sp, pose, nullptr, nullptr, nullptr, tau, nullptr, s);
  if (rc == WB_OK)
    rc = wb_self_collision_dir(robot, B, pose, sph, dmin, worst, wdiff, nullptr, nullptr, s);
  if (rc != WB_OK) return rc;
  float best_f = 1e30f, best_b = 1e30f;
  wb_tune bf = cands[0], bb = cands[0];
  for (const wb_tune& t : cands) {
    auto run_f = [&]() {
      return wb_eval_spline(robot, &sp, pose, nullptr, nullptr, nullptr, tau, &t, s);
    };
    auto run_b = [&]() {
      return wb_eval_backward_spline_cost_dir(robot, &sp, worst, wdiff, nullptr, nullptr, tau,
                                              dmin, lim, lim + D.d, w, cost, gq, gqd, gqdd, &t,
                                              s);
    };
    if (run_f() == WB_OK) {
      const float m = clk.time(run_f);
      if (m < best_f) {
        best_f = m;
        bf = t;
      }
    }
    if (run_b() == WB_OK) {
      // after the forward sweep and the pair stage that precede it in a step
      // (they rewrite the torques, minima, worst pairs and centre
      // differences the backward reads with the same values)
      auto pre_b = [&]() {
        wb_eval_spline(robot, &sp, pose, nullptr, nullptr, nullptr, tau, nullptr, s);
        wb_self_collision_dir(robot, B, pose, sph, dmin, worst, wdiff, nullptr, nullptr, s);
      };
      const float m = clk.time(run_b, pre_b);
      if (m < best_b) {
        best_b = m;
        bb = t;
      }
    }
  }
  cudaStreamSynchronize(s);
  if (best_f >= 1e30f || best_b >= 1e30f) {
    const std::string why = g_err.empty() ? std::string("no sweep shape applies") : g_err;
    return fail(WB_EINVAL, "%s", why.c_str());
  }
  g_err.clear();
  *fwd = bf;
  *bwd = bb;
  if (fwd_ms) *fwd_ms = best_f;
  if (bwd_ms) *bwd_ms = best_b;
  return WB_OK;
}

// Autotuner of an uneven batch: times, on the batch's own packed sizes with
// deterministic states and upstream gradients, the sweep passes for every
// per-robot choice of 1 or 2 segments (all combinations of the robots that
// have a 2-segment plan and a problem, up to 4 of them; beyond that one pass
// of coordinate descent from the defaults) in blocks of 64, 128 and 256
// threads, and the pair pass with 2, 4 and 8 warps a block (as many as fit),
// each 5 times after an L2 flush (median), and keeps the fastest for the
// batch's later calls.
extern "C" int wb_batch_autotune(wb_batch* batch, wb_batch_tune* tune, int32_t* fwd_segments,
                                 int32_t* bwd_segments, float* fwd_ms, float* bwd_ms) {
  g_err.clear();
  if (!batch) return fail(WB_EINVAL, "batch is NULL");
  const wb_batch_sizes z = batch->sizes;
  const int nr = (int)batch->robots.size();
  float best[2] = {0.0f, 0.0f}, best_pair = 0.0f;
  if (z.configs > 0) {
    DeviceGuard guard(batch->device);
    Scratch sc;
    float* q = sc.get<float>(z.joint_elems);
    float* qd = sc.get<float>(z.joint_elems);
    float* qdd = sc.get<float>(z.joint_elems);
    float* tau = sc.get<float>(z.joint_elems);
    float* gtau = sc.get<float>(z.joint_elems);
    float* gq = sc.get<float>(z.joint_elems);
    float* gqd = sc.get<float>(z.joint_elems);
    float* gqdd = sc.get<float>(z.joint_elems);
    float* pose = sc.get<float>(z.pose_elems);
    float* gpose = sc.get<float>(z.pose_elems);
    float* sph = sc.get<float>(z.sphere_elems);
    float* gsph = sc.get<float>(z.sphere_elems);
    float* dmin = sc.get<float>(z.configs);
    float* gdmin = sc.get<float>(z.configs);
    int32_t* worst = sc.get<int32_t>(z.configs);
    if (!q || !qd || !qdd || !tau || !gtau || !gq || !gqd || !gqdd || !pose || !gpose || !sph ||
        !gsph || !dmin || !gdmin || !worst)
      return fail(WB_ECUDA, "batch autotune scratch");
    {  // deterministic states: q in [-pi, pi], rates in [-2, 2] and [-5, 5], grads in [-1, 1]
      const int64_t most = std::max({z.joint_elems, z.pose_elems, z.sphere_elems, z.configs});
      std::vector<float> h((size_t)most);
      uint64_t st = 0xD1B54A32D192ED03ull;
      auto fill = [&](float* dst, int64_t n, float scale) {
        for (int64_t i = 0; i < n; ++i) {
          st = st * 6364136223846793005ull + 1442695040888963407ull;
          h[(size_t)i] = scale * ((float)((st >> 40) * (1.0 / 16777216.0)) * 2.0f - 1.0f);
        }
        return cudaMemcpy(dst, h.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
      };
      cudaError_t e = fill(q, z.joint_elems, 3.14159265f);
      if (e == cudaSuccess) e = fill(qd, z.joint_elems, 2.0f);
      if (e == cudaSuccess) e = fill(qdd, z.joint_elems, 5.0f);
      if (e == cudaSuccess) e = fill(gtau, z.joint_elems, 1.0f);
      if (e == cudaSuccess) e = fill(gpose, z.pose_elems, 1.0f);
      if (e == cudaSuccess) e = fill(gsph, z.sphere_elems, 1.0f);
      if (e == cudaSuccess) e = fill(gdmin, z.configs, 1.0f);
      if (e != cudaSuccess) return cuda_fail(e, "batch autotune inputs");
    }
    TuneClock clk;
    if (!clk.init(sc, batch->device)) return fail(WB_ECUDA, "batch autotune stream/events");
    cudaStream_t s = clk.s;
    int* counters = const_cast<int*>(batch->d_counters);
    BatchIO io{q, qd, qdd, pose, sph, dmin, worst, tau, gpose, gsph, gdmin, gtau, gq, gqd, gqdd};
    auto sweep = [&](int pass) -> int {
      int grid = 1, rc;
      if ((rc = batch_grid_tree(batch, pass == 0, &grid))) return rc;
      cudaError_t e =
          pass == 0
              ? launch_batch_tree_fwd(batch->d_robots, batch->d_probs, batch->d_titems[0],
                                      batch->n_titems[0], counters, io, grid, batch->ns_max,
                                      batch->threads[0], s)
              : launch_batch_tree_bwd(batch->d_robots, batch->d_probs, batch->d_titems[1],
                                      batch->n_titems[1], counters + 2, io, grid, batch->ns_max,
                                      batch->threads[1], s);
      return e == cudaSuccess ? WB_OK : cuda_fail(e, "batch autotune launch");
    };
    // robots whose segments are a choice: a 2-segment plan and some problem
    std::vector<int> used(nr, 0), free_r;
    for (const BatchProblemDev& pb : batch->probs)
      if (pb.H > 0) used[pb.robot] = 1;
    for (int i = 0; i < nr; ++i)
      if (used[i] && (batch->robots[i]->dev.seg_ok & 1)) free_r.push_back(i);
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<int> cur = batch->seg[pass], bseg = cur;
      int bthr = batch->threads[pass];
      float bt = 1e30f;
      auto trial = [&](const std::vector<int>& seg) -> int {
        batch->seg[pass] = seg;
        int rc = batch_upload_items(batch, pass);
        if (rc) return rc;
        for (int thr : {64, 128, 256}) {
          batch->threads[pass] = thr;
          if (sweep(pass) != WB_OK) {  // a block that does not fit is not a candidate
            g_err.clear();
            cudaGetLastError();
            continue;
          }
          const float m = clk.time([&]() { return sweep(pass); });
          if (m < bt) {
            bt = m;
            bseg = seg;
            bthr = thr;
          }
        }
        return WB_OK;
      };
      int rc;
      if (free_r.size() <= 4) {
        for (int mask = 0; mask < (1 << free_r.size()); ++mask) {
          std::vector<int> seg = cur;
          for (size_t k = 0; k < free_r.size(); ++k) seg[free_r[k]] = (mask >> k) & 1 ? 2 : 1;
          if ((rc = trial(seg))) return rc;
        }
      } else {
        if ((rc = trial(cur))) return rc;
        for (int i : free_r) {
          std::vector<int> seg = bseg;
          seg[i] = 3 - seg[i];
          if ((rc = trial(seg))) return rc;
        }
      }
      if (bt >= 1e30f) return fail(WB_ETOOBIG, "no batch sweep shape fits");
      batch->seg[pass] = bseg;
      batch->threads[pass] = bthr;
      if ((rc = batch_upload_items(batch, pass))) return rc;
      best[pass] = bt;
    }
    // the pair pass on the poses of the tuned forward sweep
    int rc;
    if ((rc = sweep(0))) return rc;
    if (batch->n_pitems > 0) {
      const int most = warps_that_fit(0, batch_pair_smem(batch->ws_words, batch->rad_words, 1));
      float bp = 1e30f;
      int bw = 0;
      for (int w : {2, 4, 8}) {
        if (w > most) continue;
        int bps = 0;
        if (batch_pair_max_blocks_per_sm(w, batch->ws_words, batch->rad_words, &bps) !=
                cudaSuccess ||
            bps < 1) {
          cudaGetLastError();
          continue;
        }
        const int grid = std::min((batch->n_pitems + w - 1) / w, bps * batch->num_sms);
        auto run = [&]() {
          return launch_batch_pair(batch->d_robots, batch->d_scheds, batch->d_probs,
                                   batch->d_pitems, batch->n_pitems, counters + 1, io, grid, w,
                                   batch->ws_words, batch->rad_words, s);
        };
        if (run() != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        const float m = clk.time(run);
        if (m < bp) {
          bp = m;
          bw = w;
        }
      }
      batch->pair_warps = bw;
      best_pair = bp < 1e30f ? bp : 0.0f;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
  }
  g_err.clear();
  wb_batch_get_tune(batch, tune, fwd_segments, bwd_segments);
  if (fwd_ms) *fwd_ms = best[0] + best_pair;
  if (bwd_ms) *bwd_ms = best[1];
  return WB_OK;
}
