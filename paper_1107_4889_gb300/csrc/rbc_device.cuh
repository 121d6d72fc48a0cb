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


}  // namespace rbc
