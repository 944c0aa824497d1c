// D3Q19 fused step of the self-tuning-EOS multiphase lattice Boltzmann model
// (Huang, Wu & Adams, arXiv:1809.02390, extended to three dimensions): lattice
// constants, collision constants, the node collision and the z-marching step
// kernel.  Included by lbm3d.cu (one translation unit).
//
// One launch per time step: each block owns a 32 x 4 column of the x-y plane and
// marches through a chunk of up to 32 z-planes.  For every plane it pulls the
// populations of its nodes (pull streaming, supplement Eq. 2), sums them into the
// density and puts the density, with a one-node ring in x and y, into a
// three-plane ring buffer in shared memory; the collision of plane z runs once
// plane z + 1 is there, so the force stencil (Eq. 12) of every node reads its 18
// neighbours' densities from shared memory.  In FP32 the populations stay in
// registers and the pulls of plane z + 2 are in flight while plane z collides; in
// FP64 the populations of the plane being collided are read again from L1/L2 (to
// keep the register count down).  Each population crosses DRAM once per step in
// each direction.
#pragma once

#include <cuda_runtime.h>

#include "lbm.h"

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
// Neighbour coordinates are precomputed with periodic wrap.  N: the node count,
// the stride between population planes, in the type S of the plane offsets (int
// when 19 N < 2^31, else long long; node indices are int).
template <typename T, typename S>
__device__ __forceinline__ void pull19(const T* __restrict__ f, S N, int nx, int ny, int xm, int x, int xp, int ym,
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
template <typename T, typename S>
__device__ __forceinline__ void stencil_collide_store(const C3<T>& c, const T (*a)[HX], const T (*b)[HX],
                                                      const T (*e)[HX], int ly, int lx, const T* fc, T* __restrict__ fout,
                                                      S N, int idx) {
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
template <typename T, bool KEEP, typename S>
__global__ void __launch_bounds__(TX* TY, KEEP ? 3 : 4)
    k_d3_step(const T* __restrict__ fin, T* __restrict__ fout, int nx, int ny, int nz, int tz, C3<T> c) {
  __shared__ T pl[3][HY][HX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, nz);
  const S N = S(nx) * ny * nz;
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

}  // namespace
