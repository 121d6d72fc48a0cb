// rbc_device.cuh -- device-side building blocks of the sm_103a library:
// the D3Q19 velocity set in the library's own ordering, the four-point
// shape-function factor, quaternion algebra and the Gay-Berne pair.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rbc {

// ---------------------------------------------------------------------------
// D3Q19 (Sec. 2.1).  Library ordering: speeds are grouped by the source row
// (c_z, c_y) they are pulled from, three per in-plane row and five per
// off-plane row:
//   p  0- 2: (0,0,0) (+1,0,0) (-1,0,0)
//   p  3- 5: (0,+1,0) (+1,+1,0) (-1,+1,0)
//   p  6- 8: (0,-1,0) (+1,-1,0) (-1,-1,0)
//   p  9-13: (0,0,+1) (+1,0,+1) (-1,0,+1) (0,+1,+1) (0,-1,+1)
//   p 14-18: (0,0,-1) (+1,0,-1) (-1,0,-1) (0,+1,-1) (0,-1,-1)
// ---------------------------------------------------------------------------
constexpr int kQ = 19;
constexpr uint32_t kXP = (1u << 1) | (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15);
constexpr uint32_t kXM = (1u << 2) | (1u << 5) | (1u << 8) | (1u << 11) | (1u << 16);
constexpr uint32_t kYP = (1u << 3) | (1u << 4) | (1u << 5) | (1u << 12) | (1u << 17);
constexpr uint32_t kYM = (1u << 6) | (1u << 7) | (1u << 8) | (1u << 13) | (1u << 18);
constexpr uint32_t kZP = 0x1Fu << 9;
constexpr uint32_t kZM = 0x1Fu << 14;

__host__ __device__ constexpr int cx(int p) { return int((kXP >> p) & 1u) - int((kXM >> p) & 1u); }
__host__ __device__ constexpr int cy(int p) { return int((kYP >> p) & 1u) - int((kYM >> p) & 1u); }
__host__ __device__ constexpr int cz(int p) { return int((kZP >> p) & 1u) - int((kZM >> p) & 1u); }
__host__ __device__ constexpr int c2(int p) { return cx(p) * cx(p) + cy(p) * cy(p) + cz(p) * cz(p); }
__host__ __device__ constexpr float wq(int p)
{
    return c2(p) == 0 ? 1.0f / 3.0f : (c2(p) == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr int opp(int p)
{
    int r = -1;
    for (int q = 0; q < kQ; ++q)
        if (cx(q) == -cx(p) && cy(q) == -cy(p) && cz(q) == -cz(p)) r = q;
    return r;
}

// compile-time checks of the velocity set: 19 distinct speeds, opposites,
// isotropy up to second order with c^2 = 1/3
constexpr bool lattice_ok()
{
    double s0 = 0, s1x = 0, sxx = 0, syy = 0, szz = 0, sxy = 0;
    for (int p = 0; p < kQ; ++p) {
        if (opp(p) < 0 || opp(opp(p)) != p) return false;
        for (int q = p + 1; q < kQ; ++q)
            if (cx(p) == cx(q) && cy(p) == cy(q) && cz(p) == cz(q)) return false;
        double w = c2(p) == 0 ? 1.0 / 3.0 : (c2(p) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        s0 += w;
        s1x += w * cx(p);
        sxx += w * cx(p) * cx(p);
        syy += w * cy(p) * cy(p);
        szz += w * cz(p) * cz(p);
        sxy += w * cx(p) * cy(p);
    }
    auto near = [](double a, double b) { return a - b < 1e-12 && b - a < 1e-12; };
    return near(s0, 1.0) && near(s1x, 0.0) && near(sxx, 1.0 / 3.0) && near(syy, 1.0 / 3.0) &&
           near(szz, 1.0 / 3.0) && near(sxy, 0.0);
}
static_assert(lattice_ok(), "D3Q19 velocity set");

// ---------------------------------------------------------------------------
// Shape function factor (Sec. 2.2): Peskin's four-point kernel of r = 2|y|/xi
// (support |y| <= xi; the printed branches are read as this kernel).
// ---------------------------------------------------------------------------
// Both radicands are >= 1 on their branch (1 + 4r - 4r^2 on [0, 1],
// -7 + 12r - 4r^2 on [1, 2]), so sqrt(x) = x rsqrt(x) needs no special case.
__device__ __forceinline__ float peskin4(float r)
{
    r = fabsf(r);
    if (r >= 2.0f) return 0.0f;
    const bool inner = r <= 1.0f;
    const float x = inner ? 1.0f + 4.0f * r - 4.0f * r * r : -7.0f + 12.0f * r - 4.0f * r * r;
    const float root = x * rsqrtf(x);
    return 0.125f * (inner ? 3.0f - 2.0f * r + root : 5.0f - 2.0f * r - root);
}

// ---------------------------------------------------------------------------
// Rotations.  q = (w, x, y, z) maps body to lab; Q columns are the body axes.
// ---------------------------------------------------------------------------
__host__ __device__ inline void quat_matrix(const double q[4], double Q[9])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    Q[0] = 1.0 - 2.0 * (y * y + z * z);
    Q[1] = 2.0 * (x * y - w * z);
    Q[2] = 2.0 * (x * z + w * y);
    Q[3] = 2.0 * (x * y + w * z);
    Q[4] = 1.0 - 2.0 * (x * x + z * z);
    Q[5] = 2.0 * (y * z - w * x);
    Q[6] = 2.0 * (x * z - w * y);
    Q[7] = 2.0 * (y * z + w * x);
    Q[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Symmetric 3x3 matrix: xx yy zz xy xz yz.
struct Sym3 {
    double xx, yy, zz, xy, xz, yz;
};

// A = Q diag(a^2) Q^T (Sec. 2.5)
__host__ __device__ inline Sym3 shape_tensor(const double Q[9], const double a2[3])
{
    Sym3 A;
    A.xx = Q[0] * Q[0] * a2[0] + Q[1] * Q[1] * a2[1] + Q[2] * Q[2] * a2[2];
    A.yy = Q[3] * Q[3] * a2[0] + Q[4] * Q[4] * a2[1] + Q[5] * Q[5] * a2[2];
    A.zz = Q[6] * Q[6] * a2[0] + Q[7] * Q[7] * a2[1] + Q[8] * Q[8] * a2[2];
    A.xy = Q[0] * Q[3] * a2[0] + Q[1] * Q[4] * a2[1] + Q[2] * Q[5] * a2[2];
    A.xz = Q[0] * Q[6] * a2[0] + Q[1] * Q[7] * a2[1] + Q[2] * Q[8] * a2[2];
    A.yz = Q[3] * Q[6] * a2[0] + Q[4] * Q[7] * a2[1] + Q[5] * Q[8] * a2[2];
    return A;
}

__device__ __forceinline__ void sym_apply(const Sym3 &A, const double v[3], double r[3])
{
    r[0] = A.xx * v[0] + A.xy * v[1] + A.xz * v[2];
    r[1] = A.xy * v[0] + A.yy * v[1] + A.yz * v[2];
    r[2] = A.xz * v[0] + A.yz * v[1] + A.zz * v[2];
}

// ---------------------------------------------------------------------------
// Gay-Berne pair (Sec. 2.5, App. B), d = R_i - R_j: the force on i and the
// lab-frame torque on i; returns true if the pair is inside the range.
//   kappa = (A_i + A_j)^-1 d, phi = (d.kappa) / (2 R^2), sigma = phi^-1/2,
//   rho = (R - sigma + sigma_min) / sigma_min, range rho <= 2^(1/6),
//   F_i = -u'(rho)/sigma_min d^ - (du/dphi / R^2) (kappa - (kappa.d^) d^),
//   du/dphi = u'(rho) sigma^3 / (2 sigma_min),
//   tau_i = (-A_i kappa) x f_kappa, f_kappa = -(du/dphi / R^2) kappa.
// rho below rho_floor is evaluated at rho_floor and counted.
// ---------------------------------------------------------------------------
// Precision: the geometry -- kappa, R, phi, sigma, rho -- and u'(rho) in
// FP64, so the range test and the clamp count are exact and the two
// differences of nearly equal numbers (the gap R - sigma, and u'(rho) near
// the minimum of the potential) keep FP64 accuracy; the force and torque
// vectors in FP32 from them (relative error ~1e-7).  F and T are this pair's
// contribution; the caller sums them per cell in FP64.  Ai_f: A_i in FP32
// (xx yy zz xy xz yz); ismin = 1 / sigma_min.
__device__ inline bool gb_pair_mixed(const double d[3], const Sym3 &Ai, const Sym3 &Aj, const float Ai_f[6],
                                     double smin, double ismin, double eps0, double rho_floor, double rho_cut,
                                     float F[3], float T[3], int &clamped)
{
    Sym3 H{Ai.xx + Aj.xx, Ai.yy + Aj.yy, Ai.zz + Aj.zz, Ai.xy + Aj.xy, Ai.xz + Aj.xz, Ai.yz + Aj.yz};
    const double cxx = H.yy * H.zz - H.yz * H.yz;
    const double cyy = H.xx * H.zz - H.xz * H.xz;
    const double czz = H.xx * H.yy - H.xy * H.xy;
    const double cxy = H.xz * H.yz - H.xy * H.zz;
    const double cxz = H.xy * H.yz - H.xz * H.yy;
    const double cyz = H.xy * H.xz - H.xx * H.yz;
    const double idet = 1.0 / (H.xx * cxx + H.xy * cxy + H.xz * cxz);
    double k[3];
    k[0] = (cxx * d[0] + cxy * d[1] + cxz * d[2]) * idet;
    k[1] = (cxy * d[0] + cyy * d[1] + cyz * d[2]) * idet;
    k[2] = (cxz * d[0] + cyz * d[1] + czz * d[2]) * idet;
    const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double R = sqrt(R2);
    const double phi = 0.5 * (d[0] * k[0] + d[1] * k[1] + d[2] * k[2]) / R2;
    const double sigma = 1.0 / sqrt(phi);
    double rho = (R - sigma + smin) / smin;
    if (rho > rho_cut) return false;
    if (rho < rho_floor) {
        rho = rho_floor;
        clamped++;
    }
    // u'(rho) in FP64 too: 2 rho^-13 - rho^-7 cancels near the minimum of
    // the potential
    const double ir = 1.0 / rho;
    const double ir2 = ir * ir;
    const double ir6 = ir2 * ir2 * ir2;
    const double ir7 = ir6 * ir;
    const double ir13 = ir6 * ir7;
    const double dud = -24.0 * eps0 * (2.0 * ir13 - ir7);  // du/drho
    const float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
    const float kf[3] = {(float)k[0], (float)k[1], (float)k[2]};
    const float Rf = (float)R, R2f = (float)R2;
    const float dudR = (float)(dud * ismin);
    const float dudphi = (float)(dud * sigma * sigma * sigma * (0.5 * ismin));
    const float iR = 1.0f / Rf;
    const float kR = (kf[0] * df[0] + kf[1] * df[1] + kf[2] * df[2]) * iR;
    const float g = dudphi / R2f;
    float fk[3];
    for (int a = 0; a < 3; ++a) {
        F[a] = -dudR * df[a] * iR - g * (kf[a] - kR * df[a] * iR);
        fk[a] = -g * kf[a];
    }
    const float Ak[3] = {Ai_f[0] * kf[0] + Ai_f[3] * kf[1] + Ai_f[4] * kf[2],
                         Ai_f[3] * kf[0] + Ai_f[1] * kf[1] + Ai_f[5] * kf[2],
                         Ai_f[4] * kf[0] + Ai_f[5] * kf[1] + Ai_f[2] * kf[2]};
    // (-A_i kappa) x f_kappa
    T[0] = -(Ak[1] * fk[2] - Ak[2] * fk[1]);
    T[1] = -(Ak[2] * fk[0] - Ak[0] * fk[2]);
    T[2] = -(Ak[0] * fk[1] - Ak[1] * fk[0]);
    return true;
}

}  // namespace rbc
