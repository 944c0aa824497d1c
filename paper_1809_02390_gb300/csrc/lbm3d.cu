// D3Q19 form of the self-tuning-EOS multiphase lattice Boltzmann time step
// (Huang, Wu & Adams, arXiv:1809.02390, extended to three dimensions) and the
// lb_d3_* C ABI of include/lbm3d.h.
//
// One launch per time step: each block owns a 32 x 4 column of the x-y plane and
// marches through 32 z-planes.  For every plane it pulls the populations of its
// nodes (pull streaming, supplement Eq. 2), sums them into the density and puts
// the density, with a one-node ring in x and y, into a three-plane ring buffer
// in shared memory; the collision of plane z runs once plane z + 1 is there, so
// the force stencil (Eq. 12) of every node reads its 18 neighbours' densities
// from shared memory.  In FP32 the populations stay in registers and the pulls of
// plane z + 2 are in flight while plane z collides; in FP64 the populations of
// the plane being collided are read again from L1/L2 (to keep the register count
// down).  Each population crosses DRAM once per step in each direction.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm3d.h"
#include "lbm_internal.h"

namespace {

constexpr int Q = 19;
// Plane order: rest, +x -x, +y -y, +z -z, then six opposite pairs of edge
// velocities; plane 2P + 1 is the + member of pair P (P = 0..8) and 2P + 2 its
// opposite.  Pair directions: x, y, z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1),
// (0,1,1), (0,1,-1).
constexpr int kEX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kEY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int kEZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
// The same velocities for the moments kernel.
__constant__ int cEX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int cEY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int cEZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

constexpr int TX = 32, TY = 4, TZ = 32;  // TZ: the longest z-chunk (see chunk_planes)
constexpr int HX = TX + 2, HY = TY + 2;
constexpr int kRing = 2 * HX + 2 * TY;  // ring slots of one density plane (76)
static_assert(kRing <= TX * TY, "every ring slot needs a thread of the block");
constexpr double kSEps3 = 1.75;

// Collision constants (host: make_c3).
template <typename T>
struct C3 {
  int eos;
  T rho_ref, G2, lam_RT, lam_a, b, bq;
  T se, seps, sq, sp, sm, spi;
  T k_seps_ome;  // k s_eps (s_e/2 - 1): entry (e, eps) of S
  T h_sq_ome;    // h s_q (s_e/2 - 1): entry (e, q_a) of S divided by u_a
  T b_sq_omp;    // b s_q (s_p/2 - 1): scale of the (second order, q) entries of S
  T beta2;
};

// p_EOS / c^2 (times K_EOS / c^2): vdW rho R T/(1 - b rho) - a rho^2, or
// Carnahan-Starling (Eq. 20) with t = b rho / 4.
template <typename T>
__device__ __forceinline__ T p_eos(const C3<T>& c, T rho) {
  if (c.eos == LB_EOS_VDW) return c.lam_RT * rho / (T(1) - c.b * rho) - c.lam_a * rho * rho;
  const T t = c.bq * rho;
  const T om = T(1) - t;
  const T z = (T(1) + t * (T(1) + t * (T(1) - t))) / (om * om * om);
  return c.lam_RT * rho * z - c.lam_a * rho * rho;
}

// Post-collision populations o (deviations from w_i rho_ref) of one node from
// its post-streaming deviations f, its density deviation delta = rho - rho_ref
// and the force stencil sum s = sum_i omega_i rho(x + e_i) e_i.  Moments are the
// D3Q19 polynomials (rho, e, eps, j, q, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz,
// p_xz, m) of the pairs' even and odd parts; the collision is
// mbar = m + F_m - S (m - m_eq + F_m/2 - Q_m) with the 3-D S, and the inverse
// uses M^-1 = M^T diag(1 / |row|^2).
template <typename T>
__device__ __forceinline__ void collide3(const C3<T>& c, const T* f, T delta, T sx, T sy, T sz, T* o) {
  T s[9], d[9];
#pragma unroll
  for (int P = 0; P < 9; ++P) {
    s[P] = f[2 * P + 1] + f[2 * P + 2];
    d[P] = f[2 * P + 1] - f[2 * P + 2];
  }
  const T rho = delta + c.rho_ref;
  const T A = s[0] + s[1] + s[2];
  const T Ed = (s[3] + s[4]) + (s[5] + s[6]) + (s[7] + s[8]);
  const T m_e = T(-30) * f[0] - T(11) * A + T(8) * Ed;
  const T m_eps = T(12) * f[0] - T(4) * A + Ed;
  const T jx = d[0] + ((d[3] + d[4]) + (d[5] + d[6]));
  const T jy = d[1] + ((d[3] - d[4]) + (d[7] + d[8]));
  const T jz = d[2] + ((d[5] - d[6]) + (d[7] - d[8]));
  const T qx = jx - T(5) * d[0], qy = jy - T(5) * d[1], qz = jz - T(5) * d[2];
  const T Xa = T(2) * s[0] - s[1] - s[2];
  const T Xe = (s[3] + s[4]) + (s[5] + s[6]) - T(2) * (s[7] + s[8]);
  const T pxx = Xa + Xe, pixx = Xe - T(2) * Xa;
  const T Wa = s[1] - s[2];
  const T We = (s[3] + s[4]) - (s[5] + s[6]);
  const T pww = Wa + We, piww = We - T(2) * Wa;
  const T pxy = s[3] - s[4], pxz = s[5] - s[6], pyz = s[7] - s[8];
  const T mx = (d[3] + d[4]) - (d[5] + d[6]);
  const T my = (d[4] - d[3]) + (d[7] + d[8]);
  const T mz = (d[5] - d[6]) - (d[7] - d[8]);

  // Force (Eq. 12), velocity (Eq. 5) and eta of the self-tuning EOS:
  // p_LBE = p_EOS + G^2 rho^2 / 2 (Eq. 18) = (rho + eta) / 3 (Eq. 9).
  const T Fx = c.G2 * rho * sx, Fy = c.G2 * rho * sy, Fz = c.G2 * rho * sz;
  const T irho = T(1) / rho;
  const T ux = (jx + T(0.5) * Fx) * irho, uy = (jy + T(0.5) * Fy) * irho, uz = (jz + T(0.5) * Fz) * irho;
  const T eta = T(3) * (p_eos(c, rho) + T(0.5) * c.G2 * rho * rho) - rho;
  const T rx = rho * ux, ry = rho * uy, rz = rho * uz;
  const T rhouu = rx * ux + ry * uy + rz * uz;
  const T Fu = Fx * ux + Fy * uy + Fz * uz;

  // G = m - m_eq + F_m / 2 (the shift w_i rho_ref folded into the equilibria).
  const T Ge = m_e + T(11) * delta - T(19) * eta - T(19) * rhouu + T(19) * Fu;
  const T Geps = m_eps - T(3) * delta + T(5.5) * rhouu - c.beta2 * eta - T(5.5) * Fu;
  const T two3 = T(2.0 / 3.0);
  const T Gqx = qx + two3 * jx, Gqy = qy + two3 * jy, Gqz = qz + two3 * jz;
  const T Dxx = T(2) * rx * ux - ry * uy - rz * uz;
  const T FDxx = T(2) * Fx * ux - Fy * uy - Fz * uz;
  const T Dww = ry * uy - rz * uz;
  const T FDww = Fy * uy - Fz * uz;
  const T Fxy = Fx * uy + Fy * ux, Fyz = Fy * uz + Fz * uy, Fxz = Fx * uz + Fz * ux;
  const T Gpxx = pxx - Dxx + FDxx;
  const T Gpixx = pixx + T(0.5) * (Dxx - FDxx);
  const T Gpww = pww - Dww + FDww;
  const T Gpiww = piww + T(0.5) * (Dww - FDww);
  const T Gpxy = pxy - rx * uy + T(0.5) * Fxy;
  const T Gpyz = pyz - ry * uz + T(0.5) * Fyz;
  const T Gpxz = pxz - rx * uz + T(0.5) * Fxz;

  // Q_m (Eq. 14 in 3-D) with F~ = G s.
  const T sxx = sx * sx, syy = sy * sy, szz = sz * sz;
  const T Q2 = c.G2 * (sxx + syy + szz);
  const T Qe = T(95.0 / 24.0) * Q2, Qeps = T(-55.0 / 48.0) * Q2;
  const T g12 = c.G2 * T(1.0 / 12.0);
  const T Qxx = g12 * (T(2) * sxx - syy - szz), Qww = g12 * (syy - szz);
  const T Qxy = g12 * sx * sy, Qyz = g12 * sy * sz, Qxz = g12 * sx * sz;

  const T bq = c.b_sq_omp;
  const T Geps_Q = Geps - Qeps;
  const T me = m_e + T(38) * Fu - c.se * (Ge - Qe) - c.k_seps_ome * Geps_Q -
               c.h_sq_ome * (ux * Gqx + uy * Gqy + uz * Gqz);
  const T meps = m_eps - T(11) * Fu - c.seps * Geps_Q;
  const T jxb = jx + Fx, jyb = jy + Fy, jzb = jz + Fz;
  const T qxb = qx - two3 * Fx - c.sq * Gqx;
  const T qyb = qy - two3 * Fy - c.sq * Gqy;
  const T qzb = qz - two3 * Fz - c.sq * Gqz;
  const T pxxb = pxx + T(2) * FDxx - c.sp * (Gpxx - Qxx) - bq * (T(4) * ux * Gqx - T(2) * (uy * Gqy + uz * Gqz));
  const T pixxb = pixx - FDxx - c.spi * (Gpixx + T(0.5) * Qxx);
  const T pwwb = pww + T(2) * FDww - c.sp * (Gpww - Qww) - bq * (T(2) * (uy * Gqy - uz * Gqz));
  const T piwwb = piww - FDww - c.spi * (Gpiww + T(0.5) * Qww);
  const T pxyb = pxy + Fxy - c.sp * (Gpxy - Qxy) - bq * (uy * Gqx + ux * Gqy);
  const T pyzb = pyz + Fyz - c.sp * (Gpyz - Qyz) - bq * (uz * Gqy + uy * Gqz);
  const T pxzb = pxz + Fxz - c.sp * (Gpxz - Qxz) - bq * (uz * Gqx + ux * Gqz);
  const T om = T(1) - c.sm;
  const T mxb = om * mx, myb = om * my, mzb = om * mz;

  // Inverse transform: scaled moments, then the rest node and the nine pairs.
  const T r_ = delta * T(1.0 / 19.0);
  const T e_ = me * T(1.0 / 2394.0), p_ = meps * T(1.0 / 252.0);
  const T jx_ = jxb * T(0.1), jy_ = jyb * T(0.1), jz_ = jzb * T(0.1);
  const T qx_ = qxb * T(1.0 / 40.0), qy_ = qyb * T(1.0 / 40.0), qz_ = qzb * T(1.0 / 40.0);
  const T xx_ = pxxb * T(1.0 / 36.0), ixx_ = pixxb * T(1.0 / 72.0);
  const T ww_ = pwwb * T(1.0 / 12.0), iww_ = piwwb * T(1.0 / 24.0);
  const T xy_ = pxyb * T(0.25), yz_ = pyzb * T(0.25), xz_ = pxzb * T(0.25);
  const T mx_ = mxb * T(0.125), my_ = myb * T(0.125), mz_ = mzb * T(0.125);
  o[0] = r_ - T(30) * e_ + T(12) * p_;
  const T ax = r_ - T(11) * e_ - T(4) * p_;
  const T ayz = ax - xx_ + T(2) * ixx_;
  {
    const T ev = ax + T(2) * xx_ - T(4) * ixx_, od = jx_ - T(4) * qx_;
    o[1] = ev + od;
    o[2] = ev - od;
  }
  {
    const T ev = ayz + ww_ - T(2) * iww_, od = jy_ - T(4) * qy_;
    o[3] = ev + od;
    o[4] = ev - od;
  }
  {
    const T ev = ayz - ww_ + T(2) * iww_, od = jz_ - T(4) * qz_;
    o[5] = ev + od;
    o[6] = ev - od;
  }
  const T ce = r_ + T(8) * e_ + p_;
  const T cx = ce + xx_ + ixx_;
  const T exy = cx + ww_ + iww_, exz = cx - ww_ - iww_, eyz = ce - T(2) * (xx_ + ixx_);
  const T JX = jx_ + qx_, JY = jy_ + qy_, JZ = jz_ + qz_;
  {
    const T ev = exy + xy_, od = JX + JY + mx_ - my_;
    o[7] = ev + od;
    o[8] = ev - od;
  }
  {
    const T ev = exy - xy_, od = JX - JY + mx_ + my_;
    o[9] = ev + od;
    o[10] = ev - od;
  }
  {
    const T ev = exz + xz_, od = JX + JZ - mx_ + mz_;
    o[11] = ev + od;
    o[12] = ev - od;
  }
  {
    const T ev = exz - xz_, od = JX - JZ - mx_ - mz_;
    o[13] = ev + od;
    o[14] = ev - od;
  }
  {
    const T ev = eyz + yz_, od = JY + JZ + my_ - mz_;
    o[15] = ev + od;
    o[16] = ev - od;
  }
  {
    const T ev = eyz - yz_, od = JY - JZ + my_ + mz_;
    o[17] = ev + od;
    o[18] = ev - od;
  }
}

// Populations arriving at node (x, y, z) (pull streaming): f_i from x - e_i.
// Neighbour coordinates are precomputed with periodic wrap.
template <typename T>
__device__ __forceinline__ void pull19(const T* __restrict__ f, int N, int nx, int ny, int xm, int x, int xp, int ym,
                                       int y, int yp, int zm, int z, int zp, T* v) {
  const int r00 = (z * ny + y) * nx, rm0 = (z * ny + ym) * nx, rp0 = (z * ny + yp) * nx;
  const int r0m = (zm * ny + y) * nx, r0p = (zp * ny + y) * nx;
  const int rmm = (zm * ny + ym) * nx, rpp = (zp * ny + yp) * nx;
  const int rmp = (zp * ny + ym) * nx, rpm = (zm * ny + yp) * nx;
  v[0] = __ldg(f + r00 + x);
  v[1] = __ldg(f + N + r00 + xm);
  v[2] = __ldg(f + 2 * N + r00 + xp);
  v[3] = __ldg(f + 3 * N + rm0 + x);
  v[4] = __ldg(f + 4 * N + rp0 + x);
  v[5] = __ldg(f + 5 * N + r0m + x);
  v[6] = __ldg(f + 6 * N + r0p + x);
  v[7] = __ldg(f + 7 * N + rm0 + xm);
  v[8] = __ldg(f + 8 * N + rp0 + xp);
  v[9] = __ldg(f + 9 * N + rp0 + xm);
  v[10] = __ldg(f + 10 * N + rm0 + xp);
  v[11] = __ldg(f + 11 * N + r0m + xm);
  v[12] = __ldg(f + 12 * N + r0p + xp);
  v[13] = __ldg(f + 13 * N + r0p + xm);
  v[14] = __ldg(f + 14 * N + r0m + xp);
  v[15] = __ldg(f + 15 * N + rmm + x);
  v[16] = __ldg(f + 16 * N + rpp + x);
  v[17] = __ldg(f + 17 * N + rmp + x);
  v[18] = __ldg(f + 18 * N + rpm + x);
}

template <typename T>
__device__ __forceinline__ T sum19(const T* v) {
  T a = v[0];
#pragma unroll
  for (int P = 0; P < 9; ++P) a += v[2 * P + 1] + v[2 * P + 2];
  return a;
}

__device__ __forceinline__ int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}
__device__ __forceinline__ int dec(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int inc(int a, int n) { return a == n - 1 ? 0 : a + 1; }

// Force stencil of node (ly, lx) from the density planes of z - 1 (a), z (b) and
// z + 1 (e), collision and store of its 19 outputs.
template <typename T>
__device__ __forceinline__ void stencil_collide_store(const C3<T>& c, const T (*a)[HX], const T (*b)[HX],
                                                      const T (*e)[HX], int ly, int lx, const T* fc, T* __restrict__ fout,
                                                      int N, int idx) {
  const T sxv = T(1.0 / 6.0) * (b[ly][lx + 1] - b[ly][lx - 1]) +
                T(1.0 / 12.0) * ((b[ly + 1][lx + 1] - b[ly - 1][lx - 1]) + (b[ly - 1][lx + 1] - b[ly + 1][lx - 1]) +
                                 (e[ly][lx + 1] - a[ly][lx - 1]) + (a[ly][lx + 1] - e[ly][lx - 1]));
  const T syv = T(1.0 / 6.0) * (b[ly + 1][lx] - b[ly - 1][lx]) +
                T(1.0 / 12.0) * ((b[ly + 1][lx + 1] - b[ly - 1][lx - 1]) + (b[ly + 1][lx - 1] - b[ly - 1][lx + 1]) +
                                 (e[ly + 1][lx] - a[ly - 1][lx]) + (a[ly + 1][lx] - e[ly - 1][lx]));
  const T szv = T(1.0 / 6.0) * (e[ly][lx] - a[ly][lx]) +
                T(1.0 / 12.0) * ((e[ly][lx + 1] - a[ly][lx - 1]) + (e[ly][lx - 1] - a[ly][lx + 1]) +
                                 (e[ly + 1][lx] - a[ly - 1][lx]) + (e[ly - 1][lx] - a[ly + 1][lx]));
  T o[Q];
  collide3(c, fc, b[ly][lx], sxv, syv, szv, o);
#pragma unroll
  for (int i = 0; i < Q; ++i) fout[i * N + idx] = o[i];
}

// The fused step.  Grid (ceil(nx/32), ceil(ny/4), ceil(nz/tz)), block (32, 4); each
// block marches a chunk of tz <= 32 planes (chunk_planes picks tz).
// Threads of ragged tiles that lie outside the lattice fill their ring-buffer
// slot with the density of the wrapped node and do not collide.
//   KEEP (FP32, 3 blocks per SM, up to 170 registers): software pipeline in
//   registers; while plane z collides, the pulls of plane z + 2 are in flight,
//   plane z + 1 is summed and held, plane z is in fc.
//   !KEEP (FP64, 4 blocks per SM): plane z + 1 is pulled and summed before the
//   collision of plane z, whose populations are read again (L1 / L2).
template <typename T, bool KEEP>
__global__ void __launch_bounds__(TX* TY, KEEP ? 3 : 4)
    k_d3_step(const T* __restrict__ fin, T* __restrict__ fout, int nx, int ny, int nz, int tz, C3<T> c) {
  __shared__ T pl[3][HY][HX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, nz);
  const int N = nx * ny * nz;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < nx && y < ny;
  const int xg = x % nx, yg = y % ny;
  const int xm = dec(xg, nx), xp = inc(xg, nx), ym = dec(yg, ny), yp = inc(yg, ny);
  // Ring slot of this thread (threads 0..75): top row, bottom row, left and right columns.
  const bool ring = tid < kRing;
  int hsx = 0, hsy = 0;
  if (tid < HX) {
    hsx = tid;
  } else if (tid < 2 * HX) {
    hsx = tid - HX;
    hsy = HY - 1;
  } else if (ring) {
    const int r = tid - 2 * HX;
    hsx = r < TY ? 0 : HX - 1;
    hsy = 1 + (r < TY ? r : r - TY);
  }
  const int hx = wrap(x0 - 1 + hsx, nx), hy = wrap(y0 - 1 + hsy, ny);
  const int hxm = dec(hx, nx), hxp = inc(hx, nx), hym = dec(hy, ny), hyp = inc(hy, ny);
  // Plane indices run from z0 - 1 to z1, at most one lattice length outside [0, nz).
  auto zwrap = [&](int zraw) { return zraw < 0 ? zraw + nz : (zraw >= nz ? zraw - nz : zraw); };
  auto pull_node = [&](int zraw, T* v) {
    const int z = zwrap(zraw), zm = dec(z, nz), zp = inc(z, nz);
    pull19(fin, N, nx, ny, xm, xg, xp, ym, yg, yp, zm, z, zp, v);
  };
  auto pull_ring = [&](int zraw, T* v) {
    const int z = zwrap(zraw), zm = dec(z, nz), zp = inc(z, nz);
    pull19(fin, N, nx, ny, hxm, hx, hxp, hym, hy, hyp, zm, z, zp, v);
  };
  auto put = [&](int slot, const T* v, const T* r) {
    pl[slot][ty + 1][tx + 1] = sum19(v);
    if (ring) pl[slot][hsy][hsx] = sum19(r);
  };

  T fc[Q], fn[Q];
  int sp = 0, sc = 1, sn = 2;
  if constexpr (KEEP) {
    T fr[Q], gn[Q], gr[Q];
    pull_node(z0 - 1, fn);
    if (ring) pull_ring(z0 - 1, fr);
    put(0, fn, fr);
    pull_node(z0, fc);
    if (ring) pull_ring(z0, fr);
    put(1, fc, fr);
    pull_node(z0 + 1, fn);
    if (ring) pull_ring(z0 + 1, fr);
    for (int z = z0; z < z1; ++z) {
      put(sn, fn, fr);
      if (z + 1 < z1) {
        pull_node(z + 2, gn);
        if (ring) pull_ring(z + 2, gr);
      }
      __syncthreads();
      if (active) stencil_collide_store(c, pl[sp], pl[sc], pl[sn], ty + 1, tx + 1, fc, fout, N, (z * ny + y) * nx + x);
      __syncthreads();
      const int t = sp;
      sp = sc;
      sc = sn;
      sn = t;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fc[i] = fn[i];
        fn[i] = gn[i];
        fr[i] = gr[i];
      }
    }
  } else {
    // One array at a time: pull, sum, then the ring slot's pull and sum.
    auto density = [&](int zraw, int slot) {
      pull_node(zraw, fn);
      pl[slot][ty + 1][tx + 1] = sum19(fn);
      if (ring) {
        pull_ring(zraw, fn);
        pl[slot][hsy][hsx] = sum19(fn);
      }
    };
    density(z0 - 1, 0);
    density(z0, 1);
    for (int z = z0; z < z1; ++z) {
      density(z + 1, sn);
      __syncthreads();
      if (active) {
        pull_node(z, fc);
        stencil_collide_store(c, pl[sp], pl[sc], pl[sn], ty + 1, tx + 1, fc, fout, N, (z * ny + y) * nx + x);
      }
      __syncthreads();
      const int t = sp;
      sp = sc;
      sc = sn;
      sn = t;
    }
  }
}

// Initial state at rest from FP64 densities: deviations of M^-1 m_eq(rho, 0).
// Invalid densities record the first offending node in bad[0] (not positive and
// finite) or bad[1] (vdW: rho >= 1/b).
template <typename T>
__global__ void k_d3_init(const double* __restrict__ rho0, T* __restrict__ f, int N, C3<double> c,
                          unsigned long long* bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double rho = rho0[n];
  if (!(rho > 0.0) || !isfinite(rho)) {
    atomicMin(bad, (unsigned long long)n);
    return;
  }
  if (c.eos == LB_EOS_VDW && !(c.b * rho < 1.0)) {
    atomicMin(bad + 1, (unsigned long long)n);
    return;
  }
  const double delta = rho - c.rho_ref;
  const double eta = 3.0 * (p_eos(c, rho) + 0.5 * c.G2 * rho * rho) - rho;
  const double r_ = delta / 19.0, e_ = (-11.0 * delta + 19.0 * eta) / 2394.0, p_ = (3.0 * delta + c.beta2 * eta) / 252.0;
  double o[Q];
  o[0] = r_ - 30.0 * e_ + 12.0 * p_;
  const double ax = r_ - 11.0 * e_ - 4.0 * p_, ce = r_ + 8.0 * e_ + p_;
  for (int i = 1; i < 7; ++i) o[i] = ax;
  for (int i = 7; i < Q; ++i) o[i] = ce;
  for (int i = 0; i < Q; ++i) f[i * N + n] = T(o[i]);
}

// rho = sum_i fbar_i + rho_ref into an FP64 array.
template <typename T>
__global__ void k_d3_rho(const T* __restrict__ f, double* __restrict__ rho, int N, double rho_ref) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double a = 0.0;
  for (int i = 0; i < Q; ++i) a += double(f[i * N + n]);
  rho[n] = a + rho_ref;
}

// rho u = sum_i e_i fbar_i - F/2 with F = G^2 rho sum_i omega_i rho(x + e_i) e_i.
template <typename T>
__global__ void k_d3_vel(const T* __restrict__ f, const double* __restrict__ rho, double* ux, double* uy, double* uz,
                         int nx, int ny, int nz, double G2) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = nx * ny * nz;
  if (n >= N) return;
  const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
  double s[3] = {0.0, 0.0, 0.0}, j[3] = {0.0, 0.0, 0.0};
  for (int i = 1; i < Q; ++i) {
    const int xx = wrap(x + cEX[i], nx), yy = wrap(y + cEY[i], ny), zz = wrap(z + cEZ[i], nz);
    const double w = (cEX[i] * cEX[i] + cEY[i] * cEY[i] + cEZ[i] * cEZ[i]) == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
    const double r = rho[(zz * ny + yy) * nx + xx];
    s[0] += w * r * cEX[i];
    s[1] += w * r * cEY[i];
    s[2] += w * r * cEZ[i];
    const double v = double(f[i * N + n]);
    j[0] += cEX[i] * v;
    j[1] += cEY[i] * v;
    j[2] += cEZ[i] * v;
  }
  const double r0 = rho[n];
  if (ux) ux[n] = (j[0] - 0.5 * G2 * r0 * s[0]) / r0;
  if (uy) uy[n] = (j[1] - 0.5 * G2 * r0 * s[1]) / r0;
  if (uz) uz[n] = (j[2] - 0.5 * G2 * r0 * s[2]) / r0;
}

}  // namespace

struct lb_d3_handle {
  lb_params p;
  lb_derived d;
  int nz;
  void* f[2];
  int cur;
  cudaStream_t stream;
  C3<double> c64;
  C3<float> c32;
  int tz;  // planes per z-chunk of the step kernel
  // Graphs of kD3GraphSteps steps starting from buffer 0 and 1 (captured on first
  // use on the handle's private stream, launched on `stream`); graph_failed: a
  // capture failed once, so plain launches are used from then on.
  cudaStream_t cstream = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  bool graph_failed = false;
  char err[512];
};

namespace {

using namespace lbm;

int fail3(lb_d3_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    std::snprintf(h->err, sizeof(h->err), "%s", buf);
  else
    set_thread_error(buf);
  return code;
}

size_t nodes(const lb_params* p, int nz) { return size_t(p->nx) * size_t(p->ny) * size_t(nz); }

// 3-D parameters: the thermodynamics of lb_derive (Eqs. 17-22 hold unchanged),
// the 3-D coefficients of Eq. 7 and the 3-D closure of Eq. 16.
int derive3(const lb_params* p, int nz, lb_derived* d, char* err, size_t n) {
  auto bad = [&](int code, const char* m) {
    std::snprintf(err, n, "%s", m);
    return code;
  };
  if (!p || !d) return bad(LB_EINVAL, "null argument");
  if (p->nx < 1 || p->ny < 1 || nz < 1) return bad(LB_EINVAL, "nx, ny and nz must be >= 1");
  if (int64_t(Q) * p->nx * p->ny * nz >= (int64_t(1) << 31))
    return bad(LB_EINVAL, "lattice too large: 19 nx ny nz must be below 2^31");
  if (p->precision == LB_FP16S) return bad(LB_ENOTSUP, "the D3Q19 step stores FP64 or FP32 populations");
  if (p->layout != LB_LAYOUT_PLANES) return bad(LB_ENOTSUP, "the D3Q19 step uses the planes layout");
  if (p->variant != LB_AUTO && p->variant != LB_FUSED) return bad(LB_ENOTSUP, "the D3Q19 step is the fused one");
  const double w = p->varpi == 0.0 ? 1.0 / 6.0 : p->varpi;
  if (!(w > 0) || w == 1.0 || std::fabs(w - 7.0 / 18.0) < 1e-12)
    return bad(LB_EINVAL, "varpi must be > 0 and not 1 or 7/18 (singular 3-D coefficients)");
  lb_params q = *p;
  q.nx = q.nx < 3 ? 3 : q.nx;
  q.ny = q.ny < 3 ? 3 : q.ny;
  q.varpi = 1.0 / 6.0;  // validated above; the 2-D coefficients are replaced below
  q.s_q = q.s_e = q.s_eps = 1.0;
  const int rc = derive(&q, d, err, n);
  if (rc != LB_OK) return rc;
  const double k = 38.0 * (1.0 - w) / 11.0;
  d->k = k;
  d->beta2 = -19.0 / k;
  d->b = 21.0 * (1.0 - w) / (5.0 * (7.0 - 18.0 * w));
  d->h = 798.0 * w * (1.0 - w) / (5.0 * (7.0 - 18.0 * w));
  const double tau_p = 1.0 / p->s_p - 0.5;
  const double tau_q = 1.0 / (12.0 * tau_p);
  const double tau_e = 1.0 / (12.0 * (1.0 + 5.0 * k / 19.0) * tau_q);
  d->s_q = p->s_q > 0 ? p->s_q : 1.0 / (tau_q + 0.5);
  d->s_e = p->s_e > 0 ? p->s_e : 1.0 / (tau_e + 0.5);
  d->s_eps = p->s_eps > 0 ? p->s_eps : kSEps3;
  auto ok = [](double s) { return s > 0.0 && s < 2.0; };
  if (!ok(d->s_q) || !ok(d->s_e) || !ok(d->s_eps)) return bad(LB_EINVAL, "relaxation rates must lie in (0, 2)");
  return LB_OK;
}

template <typename T>
C3<T> make_c3(const lb_params& p, const lb_derived& d) {
  C3<T> c;
  c.eos = p.eos;
  c.rho_ref = T(p.rho_ref);
  c.G2 = T(d.G2);
  c.lam_RT = T(d.lam * p.R_gas * d.T);
  c.lam_a = T(d.lam * p.eos_a);
  c.b = T(p.eos_b);
  c.bq = T(p.eos_b / 4.0);
  c.se = T(d.s_e);
  c.seps = T(d.s_eps);
  c.sq = T(d.s_q);
  c.sp = T(d.s_p);
  c.sm = T(d.s_q);
  c.spi = T(d.s_eps);
  c.k_seps_ome = T(d.k * d.s_eps * (d.s_e / 2.0 - 1.0));
  c.h_sq_ome = T(d.h * d.s_q * (d.s_e / 2.0 - 1.0));
  c.b_sq_omp = T(d.b * d.s_q * (d.s_p / 2.0 - 1.0));
  c.beta2 = T(d.beta2);
  return c;
}

// Planes per z-chunk: 32 (fewest halo planes) unless that leaves fewer than two
// waves of resident blocks (3 per SM); then halved down to 2, because a block walks
// its chunk plane after plane and a short grid leaves the GPU waiting on that chain.
int chunk_planes(int nx, int ny, int nz, int sms) {
  const long long xy = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  int tz = TZ;
  while (tz > 2 && xy * ((nz + tz - 1) / tz) < 2LL * 3 * sms) tz /= 2;
  return tz;
}

void launch_step(lb_d3_handle* h) {
  const lb_params& p = h->p;
  const int tz = h->tz;
  const dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (h->nz + tz - 1) / tz), block(TX, TY);
  const void* in = h->f[h->cur];
  void* out = h->f[1 - h->cur];
  if (p.precision == LB_FP64)
    k_d3_step<double, false><<<grid, block, 0, h->stream>>>(static_cast<const double*>(in), static_cast<double*>(out),
                                                            p.nx, p.ny, h->nz, tz, h->c64);
  else
    k_d3_step<float, true><<<grid, block, 0, h->stream>>>(static_cast<const float*>(in), static_cast<float*>(out),
                                                          p.nx, p.ny, h->nz, tz, h->c32);
  h->cur = 1 - h->cur;
}

constexpr int64_t kD3GraphSteps = 64;
static_assert(kD3GraphSteps % 2 == 0, "a graph must end in the buffer it starts from");

// Captures (once) the graph of kD3GraphSteps steps that starts from buffer h->cur.
// Returns false, and leaves plain launches in use, if the capture fails.
bool ensure_graph(lb_d3_handle* h) {
  const int c = h->cur;
  if (h->exec[c]) return true;
  if (h->graph_failed) return false;
  bool ok = h->cstream || cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) ok = cudaStreamBeginCapture(h->cstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaStream_t keep = h->stream;
    h->stream = h->cstream;
    for (int64_t k = 0; k < kD3GraphSteps; ++k) launch_step(h);
    h->stream = keep;
    ok = cudaStreamEndCapture(h->cstream, &h->graph[c]) == cudaSuccess && h->graph[c];
    if (ok) ok = cudaGraphInstantiate(&h->exec[c], h->graph[c], 0) == cudaSuccess;
  }
  h->cur = c;  // the captured launches flipped it an even number of times
  if (!ok) {
    cudaGetLastError();
    h->graph_failed = true;
  }
  return ok;
}

}  // namespace

extern "C" {

void lb_d3_velocities(int* ex, int* ey, int* ez) {
  for (int i = 0; i < Q; ++i) {
    if (ex) ex[i] = kEX[i];
    if (ey) ey[i] = kEY[i];
    if (ez) ez[i] = kEZ[i];
  }
}

int lb_d3_derive(const lb_params* p, int32_t nz, lb_derived* out) {
  char err[256];
  lb_derived d;
  const int rc = derive3(p, nz, &d, err, sizeof(err));
  if (rc != LB_OK) return fail3(nullptr, rc, "%s", err);
  if (!out) return fail3(nullptr, LB_EINVAL, "null output");
  *out = d;
  return LB_OK;
}

size_t lb_d3_state_bytes(const lb_params* p, int32_t nz) {
  if (!p || nz < 1) return 0;
  return Q * nodes(p, nz) * (p->precision == LB_FP64 ? 8 : 4);
}

int lb_d3_init(lb_d3_handle** out, const lb_params* p, int32_t nz, void* f_a, void* f_b, const double* rho0,
               int rho0_on_device, void* stream) {
  if (!out) return fail3(nullptr, LB_EINVAL, "null handle pointer");
  *out = nullptr;
  char err[256];
  lb_derived d;
  int rc = derive3(p, nz, &d, err, sizeof(err));
  if (rc != LB_OK) return fail3(nullptr, rc, "%s", err);
  if (!f_a || !f_b || f_a == f_b) return fail3(nullptr, LB_EINVAL, "f_a and f_b must be two distinct device buffers");
  if (!rho0) return fail3(nullptr, LB_EINVAL, "null initial density");
  const size_t N = nodes(p, nz);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto cuda_fail = [&](cudaError_t e, const char* what) {
    return fail3(nullptr, LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  lb_params q = *p;
  const double* rho_dev = rho0;
  if (!rho0_on_device) {
    cudaError_t e = cudaMemcpyAsync(f_b, rho0, N * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the initial density");
    rho_dev = static_cast<const double*>(f_b);
  }
  if (std::isnan(q.rho_ref)) {
    std::vector<double> host;
    const double* hp = rho0;
    if (rho0_on_device) {
      host.resize(N);
      cudaError_t e = cudaMemcpyAsync(host.data(), rho0, N * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "read of the initial density");
      hp = host.data();
    }
    double sum = 0.0;
    for (size_t n = 0; n < N; ++n) sum += hp[n];
    q.rho_ref = sum / double(N);
  }
  if (q.precision == LB_FP32) q.rho_ref = double(float(q.rho_ref));
  unsigned long long* bad = nullptr;
  cudaError_t e = cudaMalloc(&bad, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc of the status words");
  e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), s);
  const C3<double> c = make_c3<double>(q, d);
  const int threads = 256, blocks = int((N + threads - 1) / threads);
  if (e == cudaSuccess) {
    if (q.precision == LB_FP64)
      k_d3_init<double><<<blocks, threads, 0, s>>>(rho_dev, static_cast<double*>(f_a), int(N), c, bad);
    else
      k_d3_init<float><<<blocks, threads, 0, s>>>(rho_dev, static_cast<float*>(f_a), int(N), c, bad);
    e = cudaGetLastError();
  }
  unsigned long long first[2] = {~0ull, ~0ull};
  if (e == cudaSuccess) e = cudaMemcpyAsync(first, bad, sizeof(first), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_fail(e, "initial state");
  if (first[0] != ~0ull)
    return fail3(nullptr, LB_EINVAL, "initial density at node %llu is not positive and finite", first[0]);
  if (first[1] != ~0ull) return fail3(nullptr, LB_EINVAL, "initial density at node %llu exceeds 1/b of the vdW EOS", first[1]);
  lb_d3_handle* h = new (std::nothrow) lb_d3_handle();
  if (!h) return fail3(nullptr, LB_EINVAL, "out of host memory");
  h->p = q;
  h->d = d;
  h->nz = nz;
  h->f[0] = f_a;
  h->f[1] = f_b;
  h->cur = 0;
  h->stream = s;
  h->c64 = c;
  h->c32 = make_c3<float>(q, d);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  h->tz = chunk_planes(q.nx, q.ny, nz, sms);
  h->err[0] = 0;
  *out = h;
  return LB_OK;
}

int lb_d3_step(lb_d3_handle* h, int64_t nsteps) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (nsteps < 0) return fail3(h, LB_EINVAL, "nsteps must be >= 0");
  // Runs of kD3GraphSteps steps replay a graph, unless the caller's stream is being
  // captured itself (then the steps go into the caller's graph as plain launches).
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (h->stream != nullptr && cudaStreamIsCapturing(h->stream, &capture) != cudaSuccess) {
    cudaGetLastError();
    capture = cudaStreamCaptureStatusActive;
  }
  while (capture == cudaStreamCaptureStatusNone && nsteps >= kD3GraphSteps && ensure_graph(h)) {
    const cudaError_t e = cudaGraphLaunch(h->exec[h->cur], h->stream);
    if (e != cudaSuccess) return fail3(h, LB_ECUDA, "step graph launch: %s", cudaGetErrorString(e));
    nsteps -= kD3GraphSteps;  // an even number of steps: the state is back in the same buffer
  }
  for (int64_t k = 0; k < nsteps; ++k) launch_step(h);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "step launch: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_moments(lb_d3_handle* h, void* rho, void* ux, void* uy, void* uz) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (!rho) return fail3(h, LB_EINVAL, "rho output is required");
  const int N = int(nodes(&h->p, h->nz));
  const int threads = 256, blocks = (N + threads - 1) / threads;
  double* r = static_cast<double*>(rho);
  const void* f = h->f[h->cur];
  if (h->p.precision == LB_FP64)
    k_d3_rho<double><<<blocks, threads, 0, h->stream>>>(static_cast<const double*>(f), r, N, h->p.rho_ref);
  else
    k_d3_rho<float><<<blocks, threads, 0, h->stream>>>(static_cast<const float*>(f), r, N, h->p.rho_ref);
  if (ux || uy || uz) {
    double *a = static_cast<double*>(ux), *b = static_cast<double*>(uy), *c = static_cast<double*>(uz);
    if (h->p.precision == LB_FP64)
      k_d3_vel<double><<<blocks, threads, 0, h->stream>>>(static_cast<const double*>(f), r, a, b, c, h->p.nx, h->p.ny,
                                                          h->nz, h->d.G2);
    else
      k_d3_vel<float><<<blocks, threads, 0, h->stream>>>(static_cast<const float*>(f), r, a, b, c, h->p.nx, h->p.ny,
                                                         h->nz, h->d.G2);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "moments launch: %s", cudaGetErrorString(e));
  return LB_OK;
}

void* lb_d3_state(const lb_d3_handle* h) { return h ? h->f[h->cur] : nullptr; }

int lb_d3_get_state(lb_d3_handle* h, void* dst) {
  if (!h || !dst) return fail3(h, LB_EINVAL, "null argument");
  const cudaError_t e = cudaMemcpyAsync(dst, h->f[h->cur], lb_d3_state_bytes(&h->p, h->nz), cudaMemcpyDeviceToDevice,
                                        h->stream);
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "state copy: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_set_state(lb_d3_handle* h, const void* src) {
  if (!h || !src) return fail3(h, LB_EINVAL, "null argument");
  const cudaError_t e = cudaMemcpyAsync(h->f[h->cur], src, lb_d3_state_bytes(&h->p, h->nz), cudaMemcpyDeviceToDevice,
                                        h->stream);
  if (e != cudaSuccess) return fail3(h, LB_ECUDA, "state copy: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_d3_get_params(const lb_d3_handle* h, lb_params* out, lb_derived* derived) {
  if (!h) return fail3(nullptr, LB_EINVAL, "null handle");
  if (out) *out = h->p;
  if (derived) *derived = h->d;
  return LB_OK;
}

const char* lb_d3_last_error(const lb_d3_handle* h) { return h ? h->err : thread_error(); }

void lb_d3_free(lb_d3_handle* h) {
  if (!h) return;
  for (int c = 0; c < 2; ++c) {
    if (h->exec[c]) cudaGraphExecDestroy(h->exec[c]);
    if (h->graph[c]) cudaGraphDestroy(h->graph[c]);
  }
  if (h->cstream) cudaStreamDestroy(h->cstream);
  delete h;
}

}  // extern "C"
