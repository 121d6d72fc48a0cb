// api.cu -- host runtime behind the C ABI of include/rbc.h.
//
// The caller lends one device workspace (PyTorch's allocator in the Python
// binding); the runtime carves every buffer out of it, validates and uploads
// the problem, and captures one coupled step as two CUDA graphs on the
// caller's stream: the cell work (bin clear, k_bin, k_gb, k_cells) and the
// lattice pass (one per ping-pong parity).  rbc_step only launches graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/rbc.h"
#include "internal.h"
#include "rbc_device.cuh"

using namespace rbc;

namespace {

thread_local std::string g_thread_err;

struct Problem {
    int nx, ny, nz, N;
    long long Np;
    int per[3];
    bool any_solid;
    bool has_bc;       // open-boundary nodes
    bool need_links;   // link words: walls or open boundaries
    bool use_list;     // node-list lattice pass
    bool want_sigma;   // stress output (cells with alpha != 0, or open boundaries)
    int nfluid;
    int nwss;          // wall-adjacent fluid nodes (wall shear stress)
    int nc;
    int prec, stochastic;
    unsigned long long seed;
    Params p;
    int nb[3], nbins, bin_cap, max_nbr;
    double bin_size[3];
    int wnb[3], nwbins;
    double wbin_size[3];
    std::vector<int> wall_start, wall_xyz;
    int nw;
    int budget_blocks;
    // compact layout (Dev in internal.h)
    bool compact = false;
    int M = 0;
    std::vector<int4> rows, batches;  // batches: (first descriptor, segments | entries << 8, bytes, 0)
    std::vector<int2> pool;           // kSegDescs copy descriptors per batch segment
    int stage_bytes = 0;
    bool has_ext = false;  // cells carry an external force or torque
    std::vector<uint8_t> near;  // near_solid of the mask (host set-up only; released after rbc_init)
};

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *ptr = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return ptr;
    }
};

int fail(std::string *err, int code, const std::string &msg)
{
    if (err) *err = msg;
    g_thread_err = msg;
    return code;
}

// node index of (x, y, z), each coordinate at most one step outside the
// lattice (periodic wrap)
inline long long node(const Problem &P, int x, int y, int z)
{
    x = x < 0 ? x + P.nx : (x >= P.nx ? x - P.nx : x);
    y = y < 0 ? y + P.ny : (y >= P.ny ? y - P.ny : y);
    z = z < 0 ? z + P.nz : (z >= P.nz ? z - P.nz : z);
    return (long long)x + (long long)P.nx * ((long long)y + (long long)P.ny * z);
}

// near[n] = 1 when a solid node lies in the 3x3x3 cube around n (periodic
// wrap), by three one-axis passes; a node with near[n] = 0 has no solid link
// neighbour, so the host loops over link neighbours skip it.
std::vector<uint8_t> near_solid(const Problem &P, const uint8_t *solid)
{
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long sy = nx, sz = (long long)nx * ny, N = sz * nz;
    std::vector<uint8_t> a(solid, solid + N), b((size_t)N);
    // along x: each row on its own (the ends wrap)
    for (long long r = 0; r < N; r += nx) {
        const uint8_t *in = &a[(size_t)r];
        uint8_t *out = &b[(size_t)r];
        out[0] = in[0] | in[1 % nx] | in[nx - 1];
        for (int x = 1; x < nx - 1; ++x) out[x] = in[x - 1] | in[x] | in[x + 1];
        if (nx > 1) out[nx - 1] = in[nx - 2] | in[nx - 1] | in[0];
    }
    a.swap(b);
    // along y and z: whole contiguous lines (of nx, or nx ny, bytes) at a
    // time, the line before and the line after (periodic)
    auto pass = [&](int n, long long st) {
        for (long long base = 0; base < N; base += st * n)  // blocks of n lines
            for (int c = 0; c < n; ++c) {
                const uint8_t *cur = &a[(size_t)(base + c * st)];
                const uint8_t *lo = &a[(size_t)(base + (c > 0 ? c - 1 : n - 1) * st)];
                const uint8_t *hi = &a[(size_t)(base + (c < n - 1 ? c + 1 : 0) * st)];
                uint8_t *out = &b[(size_t)(base + c * st)];
                for (long long k = 0; k < st; ++k) out[k] = cur[k] | lo[k] | hi[k];
            }
        a.swap(b);
    };
    pass(ny, sy);
    pass(nz, sz);
    return a;
}

inline int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Row table and batches of the compact layout (Dev in internal.h).
// fl / fh: x-range of the fluid nodes of every row (y, z).  A row's span is
// the hull of the fluid ranges of the nine rows (y + dy, z + dz), |dy|,
// |dz| <= 1, widened by one node -- it holds every node a fluid node of the
// row or its neighbours reaches through a link -- rounded out to whole
// 32-byte sectors of a population plane (A = 8 FP32 or 16 two-byte
// entries); when that hull wraps around x (a neighbour row has fluid at
// x = 0 or nx - 1) the span is the whole row.  Batches of the lattice pass:
// consecutive row segments -- a segment is a row's fluid x-range [c0, c1]
// (or one run of a branched row, or a piece of a row) with its window
// [X0, X0 + W), the range widened by one and rounded out to A entries, or the
// whole row when it wraps -- whose windows together fill a stage of cap
// entries (node_bytes staged per entry); the segment that overflows a stage
// is cut there when the room left is worth a piece.  Per segment the pool
// holds kSegDescs int2: for each of its nine upstream rows (y + dy, z + dz)
// the part of that row's span inside the window (first entry, window offset,
// entry count), the segment's (y, z), its range and window, and its offset
// in the stage's planes; per batch the total bytes its copies bring (esz
// bytes per population entry of the three or one speeds pulled from that
// row, plus G / theta (cells) and the link word from the row itself).
// Returns false when a wrapping row does not fit a stage.
bool build_compact(Problem &P, const uint8_t *solid, int esz, bool cells)
{
    const int node_bytes = kQ * esz + (cells ? 16 : 0) + 4;
    const int nx = P.nx, ny = P.ny, nz = P.nz, nrows = ny * nz;
    // spans and windows start and end on whole 32-byte sectors of the
    // population planes: 8 FP32 or 16 two-byte entries
    const int A = 32 / esz;
    const int full = (nx + A - 1) / A * A;
    std::vector<int> fl((size_t)nrows, -1), fh((size_t)nrows, -1);
    bool any_wrap = false;
    for (int r = 0; r < nrows; ++r) {
        const uint8_t *row = solid + (size_t)r * nx;
        int x = 0;
        while (x < nx && row[x]) ++x;
        if (x == nx) continue;
        fl[r] = x;
        x = nx - 1;
        while (row[x]) --x;
        fh[r] = x;
        any_wrap |= fl[r] == 0 || fh[r] == nx - 1;
    }
    P.rows.assign((size_t)nrows, make_int4(0, 0, 0, 0xFFFF));
    long long off = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            int hlo = nx, hhi = -1;
            bool wraps = false;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy) {
                    const int r2 = wrapi(y + dy, ny) + ny * wrapi(z + dz, nz);
                    if (fh[r2] < 0) continue;
                    wraps |= fl[r2] == 0 || fh[r2] == nx - 1;
                    hlo = std::min(hlo, fl[r2] - 1);
                    hhi = std::max(hhi, fh[r2] + 1);
                }
            int slo = 0, shi = 0;
            if (hhi >= 0) {
                slo = wraps ? 0 : hlo / A * A;
                shi = wraps ? full : (hhi + 1 + A - 1) / A * A;
            }
            const int r = y + ny * z;
            const int fr = fh[r] >= 0 ? (fl[r] | (fh[r] << 16)) : 0xFFFF;
            P.rows[r] = make_int4((int)std::min(off, (long long)INT32_MAX), slo, shi, fr);
            off += shi - slo;
        }
    if (off >= (1LL << 31) - 64) return false;
    P.M = (int)off;
    // batches: row segments in (z, y, x) order -- a row's fluid range, or
    // each run of a branched row, or a piece of a row wider than a stage --
    // packed into stages of cap window entries.  Entries per stage (measured
    // on the 256^3 tube): FP32 populations 256 without cells (one node per
    // consumer thread; lattice pass 449 us, against 473 with 512) and 512
    // with cells (the autotuned step then runs the pass at one CTA of two
    // stages per SM, leaving room for the cell kernels beside it: 1.198 ->
    // 1.173 ms per step; 768: 1.276 ms); 16-bit populations 768 (1.212 ms
    // with 512, 1.206 with 768, 1.359 with 1024).  When a stage holds more
    // than one row, the segment that overflows it is cut there (its rest
    // opens the next batch) unless it wraps around x or the room left is
    // small; one-row FP32 stages take whole segments (cutting them filled the
    // stages, 0.85 -> 0.98, but the windows' overlap at the cuts and the
    // extra copies cost more: 449 -> 461 us).
    const int per_stage = esz == 4 ? (cells ? 2 : 1) : 3;
    const int cap = std::max(256 * per_stage, any_wrap ? full : 0);  // window entries per stage
    if ((long long)cap * node_bytes > 96 * 1024) return false;
    auto window = [&](int c0, int c1, int &X0, int &W) {
        if (c0 == 0 || c1 == nx - 1) {
            X0 = 0;
            W = full;
        } else {
            X0 = (c0 - 1) / A * A;
            W = (c1 + 2 + A - 1) / A * A - X0;
        }
    };
    struct Seg {
        int z, y, c0, c1;
    };
    std::vector<Seg> segs;
    bool fits = true;
    auto add_seg = [&](int z, int y, int c0, int c1) {
        int X0, W;
        window(c0, c1, X0, W);
        if (W <= cap) {
            segs.push_back({z, y, c0, c1});
            return;
        }
        const int L = (cap - 2 * A) / A * A;
        if (c0 == 0 || c1 == nx - 1 || L < A) {
            fits = false;
            return;
        }
        for (int a0 = c0; a0 <= c1; a0 += L) segs.push_back({z, y, a0, std::min(c1, a0 + L - 1)});
    };
    // a row whose fluid nodes form runs separated by wide solid gaps (a
    // vessel that branched) is taken one run at a time, so that neither the
    // copies nor the consumer threads cover the gap
    const int kGap = 24;
    std::vector<std::pair<int, int>> runs;
    auto runs_of = [&](int r) {
        runs.clear();
        const uint8_t *row = solid + (size_t)r * nx;
        int x = fl[r];
        while (x <= fh[r]) {
            int e = x;
            while (e + 1 <= fh[r] && !row[e + 1]) ++e;
            if (!runs.empty() && x - runs.back().second - 1 < kGap)
                runs.back().second = e;
            else
                runs.emplace_back(x, e);
            x = e + 1;
            while (x <= fh[r] && row[x]) ++x;
        }
    };
    for (int z = 0; z < nz && fits; ++z)
        for (int y = 0; y < ny && fits; ++y) {
            const int r = y + ny * z;
            if (fh[r] < 0) continue;
            runs_of(r);
            if (runs.size() > 1 && fl[r] > 0 && fh[r] < nx - 1)
                for (const auto &run : runs) add_seg(z, y, run.first, run.second);
            else
                add_seg(z, y, fl[r], fh[r]);
        }
    if (!fits) return false;
    // copy descriptors of one segment (kSegDescs int2 in the pool): for each
    // of its nine upstream rows (y + dy, z + dz) the part of that row's span
    // inside the window -- first entry, window offset | entry count << 16 --
    // then (y, z), (c0 | c1 << 16, X0 | W << 16), (plane offset, 0)
    P.batches.clear();
    P.pool.clear();
    int most = 0;
    const int kMinPiece = per_stage == 1 ? 1 << 30 : 4 * A;
    size_t i = 0;
    while (i < segs.size()) {
        const int first = (int)P.pool.size();
        int nb = 0, total = 0;
        long long bytes = 0;
        auto emit = [&](const Seg &s, int c1, int X0, int W) {
            for (int u = 0; u < 9; ++u) {
                const int dy = u % 3 - 1, dz = u / 3 - 1;
                const int4 rt = P.rows[(size_t)wrapi(s.y + dy, ny) + (size_t)ny * wrapi(s.z + dz, nz)];
                const int lo = std::max(X0, rt.y), hi = std::min(X0 + W, rt.z);
                const int cnt = std::max(0, hi - lo);
                P.pool.push_back(cnt > 0 ? make_int2(rt.x + lo - rt.y, (lo - X0) | (cnt << 16)) : make_int2(0, 0));
                const int planes = (dy == 0 || dz == 0) ? 3 : 1;
                bytes += (long long)cnt * (esz * planes + (u == 4 ? (cells ? 16 : 0) + 4 : 0));
            }
            P.pool.push_back(make_int2(s.y, s.z));
            P.pool.push_back(make_int2(s.c0 | (c1 << 16), X0 | (W << 16)));
            P.pool.push_back(make_int2(total, 0));
            total += W;
            ++nb;
        };
        while (i < segs.size() && nb < kMaxSegs) {
            Seg &s = segs[i];
            int X0, W;
            window(s.c0, s.c1, X0, W);
            if (total + W <= cap) {
                emit(s, s.c1, X0, W);
                ++i;
                continue;
            }
            const int R = cap - total;
            const int a1 = X0 + R - 2;  // window(c0, a1) is [X0, X0 + R)
            if (s.c0 > 0 && s.c1 < nx - 1 && R >= kMinPiece && a1 >= s.c0 && a1 < s.c1) {
                emit(s, a1, X0, R);
                s.c0 = a1 + 1;
            }
            break;
        }
        P.batches.push_back(make_int4(first, nb | (total << 8), (int)bytes, 0));
        most = std::max(most, total);
    }
    P.stage_bytes = (most * node_bytes + 127) / 128 * 128;
    return true;
}

int analyse(const rbc_geometry *g, const rbc_cells *c, const rbc_params *pp, Problem &P, std::string *err)
{
    if (!g || !pp) return fail(err, RBC_EINVAL, "geometry and params are required");
    if (g->nx < 3 || g->ny < 3 || g->nz < 3) return fail(err, RBC_EINVAL, "every lattice dimension must be >= 3");
    const long long N = (long long)g->nx * g->ny * g->nz;
    if (N > 1500000000LL) return fail(err, RBC_EINVAL, "lattice too large for 32-bit node indices");
    P.nx = g->nx;
    P.ny = g->ny;
    P.nz = g->nz;
    P.N = (int)N;
    P.Np = (N + 63) / 64 * 64;
    // the lattice pass addresses the 19 population planes with 32-bit offsets
    if (19LL * P.Np >= (1LL << 32)) return fail(err, RBC_EINVAL, "lattice too large (19 * nodes must stay below 2^32)");
    for (int a = 0; a < 3; ++a) P.per[a] = g->periodic[a] ? 1 : 0;
    P.any_solid = false;
    P.nfluid = (int)N;
    if (g->solid) {
        long long ns = 0;
        for (long long n = 0; n < N; ++n) ns += g->solid[n] ? 1 : 0;
        P.any_solid = ns > 0;
        P.nfluid = (int)(N - ns);
    }
    P.has_bc = false;
    if (g->node_type) {
        for (long long n = 0; n < N; ++n) {
            const int t = g->node_type[n];
            if (t != RBC_NODE_INTERIOR && t != RBC_NODE_INLET && t != RBC_NODE_OUTLET)
                return fail(err, RBC_EINVAL, "node_type must be RBC_NODE_INTERIOR, _INLET or _OUTLET");
            if (t == RBC_NODE_INTERIOR) continue;
            if (g->solid && g->solid[n]) return fail(err, RBC_EINVAL, "an open-boundary node is solid");
            P.has_bc = true;
        }
        if (P.has_bc && !(g->inlet_radius > 0.0)) return fail(err, RBC_EINVAL, "inlet_radius must be positive");
    }
    P.need_links = P.any_solid || P.has_bc;
    // a non-periodic axis must be closed by solid end planes (indices wrap)
    const int dims[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        if (P.per[a]) continue;
        if (!g->solid) return fail(err, RBC_EINVAL, "a non-periodic axis needs solid end planes");
        const int b = (a + 1) % 3, c2 = (a + 2) % 3;
        for (int e = 0; e < 2; ++e) {
            const int at = e ? dims[a] - 1 : 0;
            for (int i = 0; i < dims[b]; ++i)
                for (int j = 0; j < dims[c2]; ++j) {
                    int X[3];
                    X[a] = at;
                    X[b] = i;
                    X[c2] = j;
                    if (!g->solid[node(P, X[0], X[1], X[2])])
                        return fail(err, RBC_EINVAL, "a non-periodic axis needs solid end planes");
                }
        }
    }
    // parameters
    const rbc_params &q = *pp;
    if (!(q.tau0 > 0.5)) return fail(err, RBC_EINVAL, "tau0 must exceed 1/2");
    if (!(q.delta >= 0.0) || !(q.kappa > 0.0)) return fail(err, RBC_EINVAL, "delta >= 0 and kappa > 0 required");
    if (!(q.mass > 0.0)) return fail(err, RBC_EINVAL, "mass must be positive");
    for (int a = 0; a < 3; ++a) {
        if (!(q.inertia[a] > 0.0)) return fail(err, RBC_EINVAL, "inertia must be positive");
        if (!(q.xi[a] > 0.0) || !(q.semi_axes[a] > 0.0)) return fail(err, RBC_EINVAL, "xi and semi_axes must be positive");
    }
    if (!(q.gamma_T >= 0.0) || !(q.gamma_R >= 0.0) || !(q.eps0 >= 0.0))
        return fail(err, RBC_EINVAL, "gamma_T, gamma_R, eps0 must be >= 0");
    if (!(q.sigma_min_wall > 0.0) || !(q.wall_radius >= 0.0)) return fail(err, RBC_EINVAL, "bad wall particle");
    if (q.precision < RBC_PREC_F32 || q.precision > RBC_PREC_BF16)
        return fail(err, RBC_EINVAL, "precision must be RBC_PREC_F32, RBC_PREC_F16 or RBC_PREC_BF16");
    if (q.rounding != RBC_ROUND_STOCHASTIC && q.rounding != RBC_ROUND_NEAREST)
        return fail(err, RBC_EINVAL, "rounding must be RBC_ROUND_STOCHASTIC or RBC_ROUND_NEAREST");
    if (q.node_list < -1 || q.node_list > 1) return fail(err, RBC_EINVAL, "node_list must be -1, 0 or 1");
    if (q.layout < RBC_LAYOUT_AUTO || q.layout > RBC_LAYOUT_COMPACT)
        return fail(err, RBC_EINVAL, "layout must be RBC_LAYOUT_AUTO, RBC_LAYOUT_DENSE or RBC_LAYOUT_COMPACT");
    P.use_list = q.node_list == 1 || (q.node_list == 0 && 2LL * P.nfluid < N);
    P.prec = q.precision;
    P.stochastic = q.rounding == RBC_ROUND_STOCHASTIC ? 1 : 0;
    P.seed = (unsigned long long)q.seed;
    const int nc = c ? c->n : 0;
    if (nc < 0) return fail(err, RBC_EINVAL, "negative cell count");
    if (nc > 0 && (!c->pos || !c->quat)) return fail(err, RBC_EINVAL, "cell positions and quaternions are required");
    P.nc = nc;
    P.has_ext = nc > 0 && (c->force_ext || c->torque_ext);
    if (P.has_ext)
        for (int k = 0; k < 3 * nc; ++k)
            if ((c->force_ext && !std::isfinite(c->force_ext[k])) || (c->torque_ext && !std::isfinite(c->torque_ext[k])))
                return fail(err, RBC_EINVAL, "non-finite external force or torque");

    Params &p = P.p;
    p.wave = 0;
    p.in_c[0] = (float)g->inlet_center[0];
    p.in_c[1] = (float)g->inlet_center[1];
    p.in_ir2 = P.has_bc ? (float)(1.0 / (g->inlet_radius * g->inlet_radius)) : 0.0f;
    p.in_umax = (float)g->inlet_umax;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(g->body_force[a]) || !std::isfinite(g->body_force_wave[a]))
            return fail(err, RBC_EINVAL, "non-finite body force");
        p.gext[a] = (float)g->body_force[a];
        p.gwave[a] = (float)g->body_force_wave[a];
        if (g->body_force_wave[a] != 0.0) p.wave = 1;
        p.xi[a] = (float)q.xi[a];
        p.a2[a] = q.semi_axes[a] * q.semi_axes[a];
        p.I[a] = q.inertia[a];
        p.periodic[a] = P.per[a];
    }
    p.tau0 = (float)q.tau0;
    p.delta = (float)q.delta;
    p.kappa = (float)q.kappa;
    p.alpha = (float)q.alpha_tt;
    const double mach = q.mach_max > 0.0 ? q.mach_max : 0.3;
    p.mach2 = (float)(mach * mach);
    p.M = q.mass;
    p.iM = 1.0 / q.mass;
    for (int a = 0; a < 3; ++a) p.iI[a] = 1.0 / q.inertia[a];
    p.gT = q.gamma_T;
    p.gR = q.gamma_R;
    p.eT = std::exp(-0.5 * q.gamma_T);
    p.eR = std::exp(-0.5 * q.gamma_R);
    p.eps0 = q.eps0;
    const double amin = std::min(q.semi_axes[0], std::min(q.semi_axes[1], q.semi_axes[2]));
    const double amax = std::max(q.semi_axes[0], std::max(q.semi_axes[1], q.semi_axes[2]));
    p.smin_cc = std::sqrt(2.0 * (amin * amin + amin * amin));
    p.smin_w = q.sigma_min_wall;
    p.rw2 = q.wall_radius * q.wall_radius;
    p.rho_floor = q.rho_floor;
    p.rho_cut = std::pow(2.0, 1.0 / 6.0);
    const double rc = q.r_cut > 0.0 ? q.r_cut : std::sqrt(2.0 * (2.0 * amax * amax)) + (p.rho_cut - 1.0) * p.smin_cc;
    const double rcw = q.r_cut_wall > 0.0 ? q.r_cut_wall
                                          : std::sqrt(2.0 * (amax * amax + p.rw2)) + (p.rho_cut - 1.0) * p.smin_w;
    p.rc2 = rc * rc;
    p.rcw2 = rcw * rcw;

    // shape box: per axis at most floor(2 |xi|) + 3 nodes
    const double xin = std::sqrt(q.xi[0] * q.xi[0] + q.xi[1] * q.xi[1] + q.xi[2] * q.xi[2]);
    const int bdim = (int)std::floor(2.0 * xin) + 3;
    p.box_max = bdim * bdim * bdim;
    p.box_dim = bdim;
    // lattice points of a convex body K number at most vol(K + unit cube);
    // the support (a parallelepiped of half-extents xi_b, its row ranges
    // widened by 1e-3) plus the cube lies in the parallelepiped of
    // half-extents xi_b + sqrt(3)/2 + 0.005
    p.sup_cap = (int)std::floor((2.0 * q.xi[0] + std::sqrt(3.0) + 0.01) * (2.0 * q.xi[1] + std::sqrt(3.0) + 0.01) *
                                (2.0 * q.xi[2] + std::sqrt(3.0) + 0.01)) + 1;
    if (nc > 0) {
        if (bdim > 40) return fail(err, RBC_EINVAL, "shape-function support too large (more than 40 nodes per axis)");
        if (bdim > std::min(g->nx, std::min(g->ny, g->nz)))
            return fail(err, RBC_EINVAL, "shape-function support does not fit in the lattice");
        if (cells_smem_bytes(p) > 200u * 1024u)
            return fail(err, RBC_EINVAL, "shape-function support too large for shared memory");
        const double bin_min = std::max(rc, rcw);
        for (int a = 0; a < 3; ++a) {
            // half the box must exceed r_cut by more than the FP32 prefilter band
            if (P.per[a] && 2.0 * (rc + 0.05) >= dims[a]) return fail(err, RBC_EINVAL, "r_cut must be below half the box");
            P.nb[a] = std::max(1, (int)std::floor(dims[a] / bin_min));
            P.bin_size[a] = (double)dims[a] / P.nb[a];
        }
        for (int i = 0; i < nc; ++i)
            for (int a = 0; a < 3; ++a) {
                const double r = c->pos[3 * i + a];
                if (!std::isfinite(r)) return fail(err, RBC_EINVAL, "non-finite cell position");
                if (!P.per[a] && (r < 0.0 || r >= dims[a])) return fail(err, RBC_EINVAL, "cell outside a non-periodic box");
            }
    } else {
        P.nb[0] = P.nb[1] = P.nb[2] = 1;
        for (int a = 0; a < 3; ++a) P.bin_size[a] = dims[a];
    }
    P.nbins = P.nb[0] * P.nb[1] * P.nb[2];
    // wall-particle grid: bins no smaller than the wall candidate radius
    // (plus the FP32 prefilter's margin)
    for (int a = 0; a < 3; ++a) {
        P.wnb[a] = std::max(1, (int)std::floor(dims[a] / (rcw + 0.01)));
        P.wbin_size[a] = (double)dims[a] / P.wnb[a];
    }
    P.nwbins = P.wnb[0] * P.wnb[1] * P.wnb[2];
    P.bin_cap = q.bin_capacity > 0 ? q.bin_capacity : 32;
    P.max_nbr = q.max_neighbors > 0 ? std::min(q.max_neighbors, 128) : 64;

    // nodes within one node of a solid node: computed once, for the wall
    // particles, the wall-shear nodes and (rbc_init) the link words
    P.want_sigma = (nc > 0 && q.alpha_tt != 0.0) || P.has_bc;
    P.near.clear();
    if (P.any_solid) P.near = near_solid(P, g->solid);
    const std::vector<uint8_t> &near = P.near;
    // wall particles: solid nodes with a fluid node among their 18 links
    P.nw = 0;
    P.wall_start.assign(P.nwbins + 1, 0);
    P.wall_xyz.clear();
    if (P.any_solid && nc > 0) {
        // solid nodes with a fluid link neighbour: marked from the fluid side
        std::vector<uint8_t> wet((size_t)N, 0);
        for (int z = 0; z < P.nz; ++z)
            for (int y = 0; y < P.ny; ++y)
                for (int x = 0; x < P.nx; ++x) {
                    const long long n = (long long)x + (long long)P.nx * ((long long)y + (long long)P.ny * z);
                    if (g->solid[n] || !near[n]) continue;
                    for (int p = 1; p < kQ; ++p) {
                        const long long m = node(P, x + cx(p), y + cy(p), z + cz(p));
                        if (g->solid[m]) wet[m] = 1;
                    }
                }
        std::vector<int> xyz, bins;
        for (int z = 0; z < P.nz; ++z)
            for (int y = 0; y < P.ny; ++y)
                for (int x = 0; x < P.nx; ++x) {
                    if (!wet[(long long)x + (long long)P.nx * ((long long)y + (long long)P.ny * z)]) continue;
                    const int X[3] = {x, y, z};
                    int b[3];
                    for (int a = 0; a < 3; ++a)
                        b[a] = std::min(P.wnb[a] - 1, (int)std::floor(X[a] / P.wbin_size[a]));
                    bins.push_back(b[0] + P.wnb[0] * (b[1] + P.wnb[1] * b[2]));
                    xyz.push_back(x);
                    xyz.push_back(y);
                    xyz.push_back(z);
                }
        P.nw = (int)bins.size();
        for (int w = 0; w < P.nw; ++w) P.wall_start[bins[w] + 1]++;
        for (int b = 0; b < P.nwbins; ++b) P.wall_start[b + 1] += P.wall_start[b];
        std::vector<int> cur(P.wall_start.begin(), P.wall_start.end() - 1);
        P.wall_xyz.assign(3 * (size_t)P.nw, 0);
        for (int w = 0; w < P.nw; ++w) {
            const int at = cur[bins[w]]++;
            for (int a = 0; a < 3; ++a) P.wall_xyz[3 * at + a] = xyz[3 * w + a];
        }
    }
    P.nwss = 0;
    if (P.any_solid && P.want_sigma) {
        for (int z = 0; z < P.nz; ++z)
            for (int y = 0; y < P.ny; ++y)
                for (int x = 0; x < P.nx; ++x) {
                    const long long n = (long long)x + (long long)P.nx * ((long long)y + (long long)P.ny * z);
                    if (g->solid[n] || !near[n]) continue;
                    for (int p = 1; p < kQ; ++p)
                        if (g->solid[node(P, x + cx(p), y + cy(p), z + cz(p))]) {
                            P.nwss++;
                            break;
                        }
                }
    }
    P.budget_blocks = budget_blocks_for(P.N);
    // storage layout
    P.compact = false;
    P.rows.clear();
    P.batches.clear();
    if (q.layout != RBC_LAYOUT_DENSE && P.any_solid && P.nx <= 32760 && P.ny < (1 << 20)) {
        const bool ok = build_compact(P, g->solid, pop_bytes(P.prec), nc > 0);
        if (ok && (q.layout == RBC_LAYOUT_COMPACT || (long long)P.M * 10 <= (long long)N * 9)) {
            P.compact = true;
            P.use_list = false;
            P.need_links = true;
            P.Np = ((long long)P.M + 1 + 63) / 64 * 64;
        }
        if (!P.compact) {
            P.rows.clear();
            P.batches.clear();
            P.pool.clear();
        }
    }
    if (q.layout == RBC_LAYOUT_COMPACT && !P.compact)
        return fail(err, RBC_EINVAL, "the compact layout needs solid nodes, nx <= 32760 and rows that fit a stage");
    if (19LL * P.Np >= (1LL << 32)) return fail(err, RBC_EINVAL, "lattice too large (19 * entries must stay below 2^32)");
    return RBC_OK;
}

// Carve the device buffers (base == nullptr only measures).
size_t carve(const Problem &P, const rbc_params *q, void *base, Dev &d)
{
    Carver cv(base);
    const size_t Np = (size_t)P.Np;
    d.nx = P.nx;
    d.ny = P.ny;
    d.nz = P.nz;
    d.N = P.N;
    d.Np = P.Np;
    d.walls = P.need_links ? 1 : 0;
    d.prec = P.prec;
    d.stochastic = P.stochastic;
    d.seed = P.seed;
    d.pops[0] = cv.take<uint8_t>(19 * Np * (size_t)pop_bytes(P.prec));
    d.pops[1] = cv.take<uint8_t>(19 * Np * (size_t)pop_bytes(P.prec));
    d.U = cv.take<float4>(Np);
    d.S = P.want_sigma ? cv.take<float4>(Np) : nullptr;
    d.Syz = P.want_sigma ? cv.take<float>(Np) : nullptr;
    d.G = P.nc > 0 ? cv.take<float4>(Np) : nullptr;
    d.rho = cv.take<float>(Np);
    // node flags stay dense (the shape lists test every node of a cell's box)
    d.solid = P.any_solid ? cv.take<uint8_t>(((size_t)P.N + 63) / 64 * 64) : nullptr;
    d.links = P.need_links ? cv.take<uint32_t>(Np) : nullptr;
    d.nfluid = P.nfluid;
    d.fluid_list = P.use_list ? cv.take<uint32_t>((size_t)std::max(P.nfluid, 1)) : nullptr;
    d.compact = P.compact ? 1 : 0;
    d.M = P.compact ? P.M : P.N;
    d.zero_entry = P.compact ? P.M : 0;
    d.rows = P.compact ? cv.take<int4>((size_t)P.ny * P.nz) : nullptr;
    d.nbatches = P.compact ? (int)P.batches.size() : 0;
    d.lb_batches = P.compact ? cv.take<int4>((size_t)std::max(d.nbatches, 1)) : nullptr;
    d.lb_pool = P.compact ? cv.take<int2>(std::max(P.pool.size(), (size_t)1)) : nullptr;
    d.lb_stage_bytes = P.compact ? P.stage_bytes : 0;
    d.nwss = P.nwss;
    d.wss_node = cv.take<int>((size_t)std::max(P.nwss, 1));
    d.wss_n = cv.take<float>(3 * (size_t)std::max(P.nwss, 1));
    d.wss_acc = cv.take<double>(3 * (size_t)std::max(P.nwss, 1));
    const size_t n = (size_t)std::max(P.nc, 1);
    d.nc = P.nc;
    d.R = cv.take<double>(3 * n);
    d.q = cv.take<double>(4 * n);
    d.V = cv.take<double>(3 * n);
    d.Om = cv.take<double>(3 * n);
    d.A = cv.take<double>(6 * n);
    d.Rf = cv.take<float>(3 * n);
    d.Af = cv.take<float>(6 * n);
    d.Fm = cv.take<double>(3 * n);
    d.Tm = cv.take<double>(3 * n);
    d.ext = P.has_ext ? cv.take<double>(6 * n) : nullptr;
    d.have = cv.take<int>(n);
    d.diag = cv.take<double>(21 * n);
    d.jl = cv.take<float>(8 * n);
    d.hdr = cv.take<float>(kHdrWords * n);
    d.sp_cap = P.nc > 0 ? P.p.box_max : 1;
    for (int b = 0; b < 2; ++b) {
        d.sp_idx[b] = cv.take<int2>(n * (size_t)d.sp_cap);
        d.sp_val[b] = cv.take<float4>(n * (size_t)d.sp_cap);
        d.sp_cnt[b] = cv.take<int>(n);
        d.sp_S[b] = cv.take<float>(n);
    }
    for (int a = 0; a < 3; ++a) {
        d.nb[a] = P.nb[a];
        d.bin_size[a] = P.bin_size[a];
    }
    d.nbins = P.nbins;
    d.bin_cap = P.bin_cap;
    d.bin_count = cv.take<int>(P.nbins);
    d.bin_cells = cv.take<int>((size_t)P.nbins * P.bin_cap);
    d.cell_bin = cv.take<int>(n);
    d.max_nbr = P.max_nbr;
    d.nbr = cv.take<int>(n * P.max_nbr);
    d.nbr_count = cv.take<int>(n);
    d.nw = P.nw;
    for (int a = 0; a < 3; ++a) {
        d.wnb[a] = P.wnb[a];
        d.wbin_size[a] = P.wbin_size[a];
    }
    d.nwbins = P.nwbins;
    d.wall_start = cv.take<int>(P.nwbins + 1);
    d.wall_xyz = cv.take<int>(3 * (size_t)std::max(P.nw, 1));
    d.flags = cv.take<int>(8);
    d.lb_work = cv.take<int>(2);
    d.lb_step = cv.take<unsigned long long>(1);
    d.clamps = cv.take<unsigned long long>(1);
    d.budget_blocks = P.budget_blocks;
    d.budget_part = cv.take<double>(8 * (size_t)P.budget_blocks);
    d.budget_out = cv.take<double>(16);
    d.accum = cv.take<double>(8);
    d.profile = cv.take<double>((size_t)std::max(P.nx, std::max(P.ny, P.nz)));
    return (cv.off + 255) & ~size_t(255);
}

}  // namespace

namespace rbc {
void raise_smem_limit(const void *func, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> limit;  // (device, kernel) -> limit set
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    int &cur = limit[std::make_pair(dev, func)];
    if (bytes <= cur) return;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess) cur = bytes;
}

// lets other translation units report through rbc_last_error(NULL)
void set_thread_error(const std::string &msg) { g_thread_err = msg; }
void set_thread_error(const char *msg) { g_thread_err = msg; }
}  // namespace rbc

struct rbc_handle {
    Problem P;
    Dev d;
    cudaStream_t stream = nullptr, side = nullptr, side2 = nullptr;
    bool own_stream = false;
    // g_pro: cell list + Gay-Berne of the initial poses (run once at init);
    // g_step[parity]: the per-cell kernel, then the lattice pass on the main
    // stream alongside the next step's cell list, Gay-Berne forces and shape
    // lists on two side streams (they touch disjoint data), joined at the end;
    // g_timed[parity]: the same with three event-record nodes (before and
    // after the per-cell kernel, after the lattice pass), captured when kernel
    // timing is first turned on.  An event-record node between two kernels
    // delays the second by several microseconds, so untimed steps run
    // graphs without them.
    cudaGraphExec_t g_pro = nullptr, g_step[2] = {nullptr, nullptr}, g_timed[2] = {nullptr, nullptr};
    cudaGraph_t src[3] = {nullptr, nullptr, nullptr};  // kept: exec updates name their nodes
    cudaGraph_t src_timed[2] = {nullptr, nullptr};
    cudaGraphNode_t ev_node[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    cudaEvent_t ev_dummy[3] = {nullptr, nullptr, nullptr}, fork_ev = nullptr, join_ev = nullptr;
    cudaEvent_t join2_ev = nullptr;
    int64_t step = 0;
    int64_t wss_samples = 0;
    int64_t profile_samples = 0;
    int profile_axis = -1;
    int timing_cap = 0, timing_used = 0;
    bool lb_first = false;  // graph order of the step: lattice pass before the side kernels
    bool split = false;     // the spread as a kernel of its own, beside the side kernels
    std::vector<cudaEvent_t> ev;  // 3 per timed step: before the cell kernel, after it, after the lattice pass
    std::string err;
    int device = 0;
    std::vector<uint8_t> solid_host;
    std::vector<long long> wss_dense;  // compact layout: lattice index of every wall-shear node
};

#define RBC_CU(call)                                                                                \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(h ? &h->err : nullptr, RBC_ECUDA,                                           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

static int capture(rbc_handle *h, void (*body)(rbc_handle *, int), int arg, cudaGraphExec_t *out,
                   cudaGraphNode_t *ev_nodes, cudaGraph_t *keep)
{
    cudaGraph_t graph = nullptr;
    RBC_CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    body(h, arg);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) return fail(&h->err, RBC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    if (ev_nodes) {
        // find the event-record nodes of the three timing points
        size_t count = 0;
        cudaGraphGetNodes(graph, nullptr, &count);
        std::vector<cudaGraphNode_t> nodes(count);
        cudaGraphGetNodes(graph, nodes.data(), &count);
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t evr;
            if (cudaGraphEventRecordNodeGetEvent(nd, &evr) != cudaSuccess) continue;
            for (int k = 0; k < 3; ++k)
                if (evr == h->ev_dummy[k]) ev_nodes[k] = nd;
        }
    }
    e = cudaGraphInstantiate(out, graph, cudaGraphInstantiateFlagUseNodePriority);
    *keep = graph;
    if (e != cudaSuccess) return fail(&h->err, RBC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    if (ev_nodes && (!ev_nodes[0] || !ev_nodes[1] || !ev_nodes[2]))
        return fail(&h->err, RBC_ECUDA, "timing nodes not found in the step graph");
    return RBC_OK;
}

static void body_step(rbc_handle *h, int parity);
static thread_local bool g_capture_timed = false;  // body_step: add the timing event nodes

// (Re-)capture the two step graphs: plain, or timed (with the event nodes,
// whose handles go to ev_node).
static int capture_steps(rbc_handle *h, bool timed)
{
    cudaGraphExec_t *ex = timed ? h->g_timed : h->g_step;
    cudaGraph_t *src = timed ? h->src_timed : h->src;
    g_capture_timed = timed;
    int r = RBC_OK;
    for (int par = 0; par < 2 && r == RBC_OK; ++par) {
        if (ex[par]) cudaGraphExecDestroy(ex[par]);
        if (src[par]) cudaGraphDestroy(src[par]);
        ex[par] = nullptr;
        src[par] = nullptr;
        r = capture(h, body_step, par, &ex[par], timed ? h->ev_node[par] : nullptr, &src[par]);
    }
    g_capture_timed = false;
    return r;
}

// Cell list, Gay-Berne forces and shape lists of the initial poses (the
// shape lists of step k live in buffer k & 1).
static void body_prologue(rbc_handle *h, int)
{
    launch_bin(h->d, h->P.p, h->stream);
    launch_gb(h->d, h->P.p, h->stream);
    launch_weights(h->d, h->P.p, 0, h->stream);
}

// The side work of a step: the next step's shape lists on one side stream,
// its cell list and Gay-Berne forces on the other.
static void launch_side(rbc_handle *h, int parity)
{
    if (h->d.nc <= 0) return;
    launch_weights(h->d, h->P.p, parity ^ 1, h->side2);
    launch_bin(h->d, h->P.p, h->side);
    launch_gb(h->d, h->P.p, h->side);
}

// One coupled step.  Main stream: the per-cell kernel (sample the fields
// with this pose's shape lists, the rigid update to the new poses, spread
// the impulses with the same lists; or, split, the spread as a kernel of its
// own after it), then the lattice pass.  As soon as the new poses exist, two
// side streams build the next step's cell list and Gay-Berne forces, and its
// shape headers and shape lists (into buffer parity ^ 1); they read only the
// poses and write nothing the spread or the lattice pass reads.  The step
// ends when all three streams have.
static void body_step(rbc_handle *h, int parity)
{
    const bool cells = h->d.nc > 0;
    const bool timed = g_capture_timed;
    if (timed) cudaEventRecordWithFlags(h->ev_dummy[0], h->stream, cudaEventRecordExternal);
    const bool split = cells && h->split;
    launch_cells(h->d, h->P.p, parity, h->stream, split);
    if (cells) {
        cudaEventRecord(h->fork_ev, h->stream);
        cudaStreamWaitEvent(h->side, h->fork_ev, 0);
        cudaStreamWaitEvent(h->side2, h->fork_ev, 0);
    }
    // Default order: the side kernels go into the graph first, so their
    // blocks are dispatched before the persistent lattice pass fills the
    // SMs and the two overlap.  The autotuner also tries the lattice pass
    // first (it then runs nearly alone and the side kernels mostly after
    // it); which is faster depends on how much cell work there is.  With
    // the spread split off the per-cell kernel, the side kernels (which
    // need only the new poses) start beside it and only the lattice pass
    // waits for it.
    if (!h->lb_first) launch_side(h, parity);
    if (split) launch_spread(h->d, h->P.p, parity, h->stream);
    if (timed) cudaEventRecordWithFlags(h->ev_dummy[1], h->stream, cudaEventRecordExternal);
    launch_lb(h->d, h->P.p, parity, h->stream);
    if (h->lb_first) launch_side(h, parity);
    if (timed) cudaEventRecordWithFlags(h->ev_dummy[2], h->stream, cudaEventRecordExternal);
    if (cells) {
        cudaEventRecord(h->join_ev, h->side);
        cudaEventRecord(h->join2_ev, h->side2);
        cudaStreamWaitEvent(h->stream, h->join_ev, 0);
        cudaStreamWaitEvent(h->stream, h->join2_ev, 0);
    }
}

namespace rbc {

// Serving: `steps` coupled steps from the handle's current step, then the
// budget reduction, which adds to the handle's time-average sums once the
// pass counter has reached average_from; captured as one graph (launched
// on the handle's stream by the request server).
static thread_local int g_tick_steps = 0;
static thread_local long long g_tick_from = 0;
static void body_ticks(rbc_handle *h, int start_parity)
{
    for (int k = 0; k < g_tick_steps; ++k) body_step(h, (start_parity + k) & 1);
    launch_budget(h->d, h->P.p, (start_parity + g_tick_steps) & 1, h->stream, true, g_tick_from);
}

int capture_ticks(rbc_handle *h, int64_t steps, long long average_from, cudaGraphExec_t *out)
{
    if (steps <= 0 || steps > (1 << 20)) return fail(&h->err, RBC_EINVAL, "tick length out of range");
    g_tick_steps = (int)steps;
    g_tick_from = average_from;
    cudaGraph_t keep = nullptr;
    const int rc = capture(h, body_ticks, (int)(h->step & 1), out, nullptr, &keep);
    if (keep) cudaGraphDestroy(keep);
    return rc;
}

void advance_steps(rbc_handle *h, int64_t steps) { h->step += steps; }

const Dev &handle_dev(const rbc_handle *h) { return h->d; }
const Params &handle_params(const rbc_handle *h) { return h->P.p; }

int read_accum(rbc_handle *h, double accum[8], int flags[8])
{
    RBC_CU(cudaMemcpyAsync(accum, h->d.accum, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaMemcpyAsync(flags, h->d.flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    return RBC_OK;
}

}  // namespace rbc

extern "C" {

void rbc_default_params(rbc_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tau0 = 1.0;
    p->delta = 2.0;
    p->kappa = 20.0;
    p->gamma_T = 0.1;
    p->gamma_R = 0.1;
    p->alpha_tt = 0.04;
    p->eps0 = 0.01;
    p->xi[0] = 4.0;
    p->xi[1] = 4.0;
    p->xi[2] = 1.5;
    p->semi_axes[0] = 4.0;
    p->semi_axes[1] = 4.0;
    p->semi_axes[2] = 1.5;
    p->mass = 10.0;
    p->inertia[0] = p->inertia[1] = p->inertia[2] = 1000.0;
    p->sigma_min_wall = 0.5;
    p->wall_radius = 0.5;
    p->rho_floor = 0.75;
    p->mach_max = 0.3;
}

int rbc_workspace_size(const rbc_geometry *geom, const rbc_cells *cells, const rbc_params *params, size_t *bytes)
{
    if (!bytes) return fail(nullptr, RBC_EINVAL, "bytes is NULL");
    Problem P;
    int rc = analyse(geom, cells, params, P, nullptr);
    if (rc != RBC_OK) return rc;
    Dev d;
    *bytes = carve(P, params, nullptr, d);
    return RBC_OK;
}

int rbc_init(const rbc_geometry *geom, const rbc_cells *cells, const rbc_params *params, void *workspace,
             size_t workspace_bytes, rbc_handle **out)
{
    if (!out) return fail(nullptr, RBC_EINVAL, "out is NULL");
    *out = nullptr;
    rbc_handle *h = new (std::nothrow) rbc_handle();
    if (!h) return fail(nullptr, RBC_ENOMEM, "host allocation failed");
    int rc = analyse(geom, cells, params, h->P, &h->err);
    if (rc != RBC_OK) {
        delete h;
        return rc;
    }
    Dev probe;
    const size_t need = carve(h->P, params, nullptr, probe);
    if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "workspace must be >= %zu bytes and 256-byte aligned", need);
        fail(nullptr, RBC_ENOMEM, msg);
        delete h;
        return RBC_ENOMEM;
    }
    carve(h->P, params, workspace, h->d);
    if (h->P.any_solid) h->solid_host.assign(geom->solid, geom->solid + h->P.N);
    cudaGetDevice(&h->device);
    if (params->stream) {
        h->stream = static_cast<cudaStream_t>(params->stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            fail(nullptr, RBC_ECUDA, "stream creation failed");
            delete h;
            return RBC_ECUDA;
        }
        h->own_stream = true;
    }
    rc = [&]() -> int {
        Dev &d = h->d;
        const Problem &P = h->P;
        cudaStream_t s = h->stream;
        const size_t Np = (size_t)P.Np;
        // fluid at rest: f = w_p, i.e. zero deviations; fields zero
        // (zero bits are a zero deviation in every storage format)
        RBC_CU(cudaMemsetAsync(d.pops[0], 0, 19 * Np * pop_bytes(d.prec), s));
        RBC_CU(cudaMemsetAsync(d.pops[1], 0, 19 * Np * pop_bytes(d.prec), s));
        RBC_CU(cudaMemsetAsync(d.U, 0, Np * sizeof(float4), s));
        if (d.S) RBC_CU(cudaMemsetAsync(d.S, 0, Np * sizeof(float4), s));
        if (d.Syz) RBC_CU(cudaMemsetAsync(d.Syz, 0, Np * sizeof(float), s));
        if (d.G) RBC_CU(cudaMemsetAsync(d.G, 0, Np * sizeof(float4), s));
        RBC_CU(cudaMemsetAsync(d.rho, 0, Np * sizeof(float), s));
        std::vector<uint32_t> links;
        if (d.solid) RBC_CU(cudaMemcpyAsync(d.solid, geom->solid, (size_t)P.N, cudaMemcpyHostToDevice, s));
        std::vector<uint32_t> flist;
        std::vector<int> wnode;
        std::vector<float> wnrm;
        if (d.compact) {
            // link words of the stored entries (bit 31: solid node, or an
            // entry past the end of a whole row); wall-shear nodes in
            // storage order with their lattice indices kept on the host
            links.assign(Np, 1u << 31);
            const std::vector<uint8_t> &near = P.near;
            for (int z = 0; z < P.nz; ++z)
                for (int y = 0; y < P.ny; ++y) {
                    const int4 rt = P.rows[(size_t)y + (size_t)P.ny * z];
                    const long long row = (long long)P.nx * ((long long)y + (long long)P.ny * z);
                    for (int x = rt.y; x < std::min(rt.z, P.nx); ++x) {
                        const long long n = row + x;
                        const size_t c = (size_t)rt.x + (size_t)(x - rt.y);
                        if (geom->solid[n]) continue;
                        uint32_t m = 0u;
                        float nv[3] = {0.f, 0.f, 0.f};
                        if (!near.empty() && near[n])
                            for (int p = 1; p < kQ; ++p)
                                if (geom->solid[node(P, x + cx(p), y + cy(p), z + cz(p))]) {
                                    m |= 1u << p;
                                    nv[0] -= (float)cx(p);
                                    nv[1] -= (float)cy(p);
                                    nv[2] -= (float)cz(p);
                                }
                        if (geom->node_type && geom->node_type[n] == RBC_NODE_INLET) m |= 1u << 29;
                        if (geom->node_type && geom->node_type[n] == RBC_NODE_OUTLET) m |= 1u << 30;
                        links[c] = m;
                        if ((m & 0x7FFFEu) && P.nwss > 0) {
                            const float nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
                            wnode.push_back((int)c);
                            h->wss_dense.push_back(n);
                            for (int a = 0; a < 3; ++a) wnrm.push_back(nn > 0.f ? nv[a] / nn : 0.f);
                        }
                    }
                }
            RBC_CU(cudaMemcpyAsync(d.links, links.data(), links.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(const_cast<int4 *>(d.rows), P.rows.data(), P.rows.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(const_cast<int4 *>(d.lb_batches), P.batches.data(), P.batches.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(const_cast<int2 *>(d.lb_pool), P.pool.data(), P.pool.size() * sizeof(int2),
                                   cudaMemcpyHostToDevice, s));
        } else if (d.links) {
            // per-node link word in the library's velocity ordering: bit p set
            // when the downstream node x + c_p is solid (fluid nodes), bit 29 /
            // 30 for inlet / outlet nodes, bit 31 when x is solid
            links.assign((size_t)P.N, 0u);
            const std::vector<uint8_t> &near = P.near;
            for (int z = 0; z < P.nz; ++z)
                for (int y = 0; y < P.ny; ++y) {
                    const long long row = (long long)P.nx * ((long long)y + (long long)P.ny * z);
                    for (int x = 0; x < P.nx; ++x) {
                        const long long n = row + x;
                        if (geom->solid && geom->solid[n]) {
                            links[n] = 1u << 31;
                            continue;
                        }
                        uint32_t m = 0u;
                        float nv[3] = {0.f, 0.f, 0.f};
                        if (!near.empty() && near[n])
                            for (int p = 1; p < kQ; ++p)
                                if (geom->solid[node(P, x + cx(p), y + cy(p), z + cz(p))]) {
                                    m |= 1u << p;
                                    nv[0] -= (float)cx(p);
                                    nv[1] -= (float)cy(p);
                                    nv[2] -= (float)cz(p);
                                }
                        if (geom->node_type && geom->node_type[n] == RBC_NODE_INLET) m |= 1u << 29;
                        if (geom->node_type && geom->node_type[n] == RBC_NODE_OUTLET) m |= 1u << 30;
                        links[n] = m;
                        if ((m & 0x7FFFEu) && P.nwss > 0) {
                            const float nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
                            wnode.push_back((int)n);
                            for (int a = 0; a < 3; ++a) wnrm.push_back(nn > 0.f ? nv[a] / nn : 0.f);
                        }
                    }
                }
            RBC_CU(cudaMemcpyAsync(d.links, links.data(), links.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        }
        std::vector<uint8_t>().swap(h->P.near);  // the set-up's last use of it
        if (d.fluid_list) {
            flist.reserve((size_t)P.nfluid);
            for (long long n = 0; n < (long long)P.N; ++n)
                if (!(geom->solid && geom->solid[n])) flist.push_back((uint32_t)n);
            RBC_CU(cudaMemcpyAsync(d.fluid_list, flist.data(), flist.size() * sizeof(uint32_t),
                                   cudaMemcpyHostToDevice, s));
        }
        if (d.nwss > 0) {
            if ((int)wnode.size() != d.nwss) return fail(&h->err, RBC_EINVAL, "wall node count mismatch");
            RBC_CU(cudaMemcpyAsync(d.wss_node, wnode.data(), wnode.size() * sizeof(int), cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(d.wss_n, wnrm.data(), wnrm.size() * sizeof(float), cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemsetAsync(d.wss_acc, 0, 3 * sizeof(double) * (size_t)d.nwss, s));
        }
        RBC_CU(cudaMemsetAsync(d.flags, 0, 8 * sizeof(int), s));
        RBC_CU(cudaMemsetAsync(d.lb_work, 0, 2 * sizeof(int), s));
        RBC_CU(cudaMemsetAsync(d.lb_step, 0, sizeof(unsigned long long), s));
        RBC_CU(cudaMemsetAsync(d.accum, 0, 8 * sizeof(double), s));
        RBC_CU(cudaMemsetAsync(d.profile, 0, sizeof(double) * (size_t)std::max(P.nx, std::max(P.ny, P.nz)), s));
        RBC_CU(cudaMemsetAsync(d.clamps, 0, sizeof(unsigned long long), s));
        const int n = P.nc;
        if (n > 0) {
            const int dims[3] = {P.nx, P.ny, P.nz};
            std::vector<double> R(3 * (size_t)n), q(4 * (size_t)n), V(3 * (size_t)n, 0.0), W(3 * (size_t)n, 0.0);
            for (int i = 0; i < n; ++i) {
                for (int a = 0; a < 3; ++a) {
                    double r = cells->pos[3 * i + a];
                    if (P.per[a]) {
                        r = std::fmod(r, (double)dims[a]);
                        if (r < 0.0) r += dims[a];
                        if (r >= dims[a]) r -= dims[a];
                    }
                    R[3 * i + a] = r;
                    if (cells->vel) V[3 * i + a] = cells->vel[3 * i + a];
                    if (cells->omega_body) W[3 * i + a] = cells->omega_body[3 * i + a];
                }
                double nq = 0.0;
                for (int k = 0; k < 4; ++k) nq += cells->quat[4 * i + k] * cells->quat[4 * i + k];
                if (!(nq > 0.0) || !std::isfinite(nq)) return fail(&h->err, RBC_EINVAL, "degenerate quaternion");
                for (int k = 0; k < 4; ++k) q[4 * i + k] = cells->quat[4 * i + k] / std::sqrt(nq);
            }
            RBC_CU(cudaMemcpyAsync(d.R, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(d.q, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(d.V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            RBC_CU(cudaMemcpyAsync(d.Om, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            if (d.ext) {
                std::vector<double> E(6 * (size_t)n, 0.0);
                for (int i = 0; i < n; ++i)
                    for (int a = 0; a < 3; ++a) {
                        if (cells->force_ext) E[6 * i + a] = cells->force_ext[3 * i + a];
                        if (cells->torque_ext) E[6 * i + 3 + a] = cells->torque_ext[3 * i + a];
                    }
                RBC_CU(cudaMemcpyAsync(d.ext, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            }
            RBC_CU(cudaMemsetAsync(d.have, 0, sizeof(int) * n, s));
            RBC_CU(cudaMemsetAsync(d.diag, 0, sizeof(double) * 21 * n, s));
            RBC_CU(cudaMemsetAsync(d.Fm, 0, sizeof(double) * 3 * n, s));
            RBC_CU(cudaMemsetAsync(d.Tm, 0, sizeof(double) * 3 * n, s));
            RBC_CU(cudaMemsetAsync(d.nbr_count, 0, sizeof(int) * n, s));
            RBC_CU(cudaMemcpyAsync(d.wall_start, P.wall_start.data(), sizeof(int) * (P.nwbins + 1),
                                   cudaMemcpyHostToDevice, s));
            if (P.nw > 0)
                RBC_CU(cudaMemcpyAsync(d.wall_xyz, P.wall_xyz.data(), sizeof(int) * 3 * (size_t)P.nw,
                                       cudaMemcpyHostToDevice, s));
            const size_t smem = cells_smem_bytes(P.p);
            (void)smem;
        }
        RBC_CU(cudaStreamSynchronize(s));
        prepare_lb(h->d);
        if (n > 0) prepare_cells(h->P.p);
        RBC_CU(cudaGetLastError());
        int least = 0, greatest = 0;
        RBC_CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        h->d.side_prio = greatest;
        RBC_CU(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        RBC_CU(cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking));
        RBC_CU(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        RBC_CU(cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
        RBC_CU(cudaEventCreateWithFlags(&h->join2_ev, cudaEventDisableTiming));
        for (int k = 0; k < 3; ++k) RBC_CU(cudaEventCreate(&h->ev_dummy[k]));
        if (n > 0) {
            int r = capture(h, body_prologue, 0, &h->g_pro, nullptr, &h->src[2]);
            if (r != RBC_OK) return r;
        }
        {
            int r = capture_steps(h, false);
            if (r != RBC_OK) return r;
        }
        // cell list and Gay-Berne forces of the initial poses
        if (h->g_pro) RBC_CU(cudaGraphLaunch(h->g_pro, s));
        RBC_CU(cudaStreamSynchronize(s));
        RBC_CU(cudaGetLastError());
        return RBC_OK;
    }();
    if (rc != RBC_OK) {
        g_thread_err = h->err;
        rbc_free(h);
        return rc;
    }
    *out = h;
    return RBC_OK;
}

static int check_flags(rbc_handle *h)
{
    int flags[8];
    RBC_CU(cudaMemcpyAsync(flags, h->d.flags, sizeof flags, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    if (flags[FLAG_OVERFLOW])
        return fail(&h->err, RBC_ENOMEM,
                    std::string("capacity exceeded:") + ((flags[FLAG_OVERFLOW] & OVF_BIN) ? " cell-list bin" : "") +
                        ((flags[FLAG_OVERFLOW] & OVF_NBR) ? " neighbour list" : "") +
                        ((flags[FLAG_OVERFLOW] & OVF_BOX) ? " shape box" : ""));
    // a timed-out pass leaves part of the lattice unupdated: report the cause
    if (flags[FLAG_TIMEOUT]) return fail(&h->err, RBC_ETIMEOUT, "a bounded wait of the lattice pass ran out");
    if (flags[FLAG_UNSTABLE]) return fail(&h->err, RBC_EUNSTABLE, "NaN or |u| above the Mach guard");
    return RBC_OK;
}

int rbc_step(rbc_handle *h, int64_t n)
{
    if (!h) return fail(nullptr, RBC_EINVAL, "handle is NULL");
    if (n < 0) return fail(&h->err, RBC_EINVAL, "negative step count");
    for (int64_t k = 0; k < n; ++k) {
        const int par = (int)(h->step & 1);
        const bool timed = h->timing_used < h->timing_cap;
        if (timed) {
            // each timed launch records into its own three events
            for (int e = 0; e < 3; ++e)
                RBC_CU(cudaGraphExecEventRecordNodeSetEvent(h->g_timed[par], h->ev_node[par][e],
                                                            h->ev[3 * (size_t)h->timing_used + e]));
            RBC_CU(cudaGraphLaunch(h->g_timed[par], h->stream));
            h->timing_used++;
        } else {
            RBC_CU(cudaGraphLaunch(h->g_step[par], h->stream));
        }
        h->step++;
    }
    return RBC_OK;
}

int rbc_fields(rbc_handle *h, double *rho, double *u, double *cells_state)
{
    if (!h) return fail(nullptr, RBC_EINVAL, "handle is NULL");
    const Dev &d = h->d;
    const size_t N = (size_t)d.N, Np = (size_t)d.Np;
    const int par = (int)(h->step & 1);
    const uint8_t *solid = h->P.any_solid ? h->solid_host.data() : nullptr;
    // storage entry of lattice node k, or -1 for a solid node (compact:
    // nodes outside every row's span are solid)
    std::vector<long long> ent;
    if (d.compact) {
        ent.assign(N, -1);
        for (size_t r = 0; r < h->P.rows.size(); ++r) {
            const int4 rt = h->P.rows[r];
            for (int x = rt.y; x < std::min(rt.z, d.nx); ++x) {
                const size_t k = (size_t)d.nx * r + (size_t)x;
                if (!solid[k]) ent[k] = (long long)rt.x + (x - rt.y);
            }
        }
    }
    if (rho) {
        launch_rho(d, par, h->stream);
        const size_t nr = d.compact ? (size_t)d.M : N;
        std::vector<float> r(nr);
        RBC_CU(cudaMemcpyAsync(r.data(), d.rho, nr * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaStreamSynchronize(h->stream));
        for (size_t k = 0; k < N; ++k) {
            if (d.compact)
                rho[k] = ent[k] < 0 ? 0.0 : 1.0 + (double)r[(size_t)ent[k]];
            else
                rho[k] = (solid && solid[k]) ? 0.0 : 1.0 + (double)r[k];
        }
    }
    if (u) {
        std::vector<float4> U(Np);
        RBC_CU(cudaMemcpyAsync(U.data(), d.U, Np * sizeof(float4), cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaStreamSynchronize(h->stream));
        for (size_t k = 0; k < N; ++k) {
            const long long e = d.compact ? ent[k] : (long long)k;
            const float4 v = e < 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : U[(size_t)e];
            u[3 * k] = v.x;
            u[3 * k + 1] = v.y;
            u[3 * k + 2] = v.z;
        }
    }
    if (cells_state && d.nc > 0) {
        const size_t n = (size_t)d.nc;
        std::vector<double> R(3 * n), q(4 * n), V(3 * n), W(3 * n);
        RBC_CU(cudaMemcpyAsync(R.data(), d.R, R.size() * 8, cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaMemcpyAsync(q.data(), d.q, q.size() * 8, cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaMemcpyAsync(V.data(), d.V, V.size() * 8, cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaMemcpyAsync(W.data(), d.Om, W.size() * 8, cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaStreamSynchronize(h->stream));
        for (size_t i = 0; i < n; ++i) {
            double *o = &cells_state[13 * i];
            for (int a = 0; a < 3; ++a) {
                o[a] = R[3 * i + a];
                o[7 + a] = V[3 * i + a];
                o[10 + a] = W[3 * i + a];
            }
            for (int k = 0; k < 4; ++k) o[3 + k] = q[4 * i + k];
        }
    }
    return check_flags(h);
}

int rbc_stats(rbc_handle *h, rbc_stats_t *out)
{
    if (!h || !out) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    const int par = (int)(h->step & 1);
    launch_budget(h->d, h->P.p, par, h->stream);
    double b[16];
    int flags[8];
    unsigned long long cl = 0;
    RBC_CU(cudaMemcpyAsync(b, h->d.budget_out, sizeof b, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaMemcpyAsync(flags, h->d.flags, sizeof flags, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaMemcpyAsync(&cl, h->d.clamps, sizeof cl, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    RBC_CU(cudaGetLastError());
    out->step = h->step;
    out->mass = b[0];
    for (int a = 0; a < 3; ++a) {
        out->p_fluid[a] = b[1 + a];
        out->p_cells[a] = b[6 + a];
    }
    out->max_u = b[4];
    out->gb_clamps = (int64_t)cl;
    out->unstable = flags[FLAG_UNSTABLE] != 0 || b[5] > 0.0;
    out->overflow = flags[FLAG_OVERFLOW];
    out->power = b[9];
    if (flags[FLAG_TIMEOUT]) return fail(&h->err, RBC_ETIMEOUT, "a bounded wait of the lattice pass ran out");
    if (out->overflow) return fail(&h->err, RBC_ENOMEM, "a device capacity was exceeded");
    if (out->unstable) return fail(&h->err, RBC_EUNSTABLE, "NaN or |u| above the Mach guard");
    return RBC_OK;
}

int rbc_cell_diag(rbc_handle *h, double *out)
{
    if (!h || !out) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    if (h->d.nc == 0) return RBC_OK;
    RBC_CU(cudaMemcpyAsync(out, h->d.diag, sizeof(double) * 21 * h->d.nc, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    return RBC_OK;
}

int rbc_neighbors(rbc_handle *h, int *counts, int *lists, int max_per_cell)
{
    if (!h || !counts || (max_per_cell > 0 && !lists)) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    const int n = h->d.nc;
    if (n == 0) return RBC_OK;
    std::vector<int> L((size_t)n * h->d.max_nbr);
    RBC_CU(cudaMemcpyAsync(counts, h->d.nbr_count, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaMemcpyAsync(L.data(), h->d.nbr, sizeof(int) * L.size(), cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    int rc = RBC_OK;
    for (int i = 0; i < n; ++i) {
        if (counts[i] > max_per_cell) rc = RBC_ENOMEM;
        for (int k = 0; k < std::min(counts[i], max_per_cell); ++k)
            lists[(size_t)i * max_per_cell + k] = L[(size_t)i * h->d.max_nbr + k];
    }
    if (rc != RBC_OK) return fail(&h->err, rc, "a neighbour list is longer than max_per_cell");
    int flags[8];
    RBC_CU(cudaMemcpy(flags, h->d.flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[FLAG_OVERFLOW] & (OVF_BIN | OVF_NBR)) return fail(&h->err, RBC_ENOMEM, "cell list capacity exceeded");
    return RBC_OK;
}

int rbc_set_timing(rbc_handle *h, int capacity)
{
    if (!h || capacity < 0) return fail(h ? &h->err : nullptr, RBC_EINVAL, "bad argument");
    RBC_CU(cudaStreamSynchronize(h->stream));
    // the timed graphs' event nodes may still name events of the previous
    // timing: point them back at the dummies before those events go
    for (int par = 0; par < 2; ++par) {
        if (!h->g_timed[par]) continue;
        for (int e = 0; e < 3; ++e)
            RBC_CU(cudaGraphExecEventRecordNodeSetEvent(h->g_timed[par], h->ev_node[par][e], h->ev_dummy[e]));
    }
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    h->timing_cap = 0;
    h->timing_used = 0;
    for (int k = 0; k < 3 * capacity; ++k) {
        cudaEvent_t e;
        RBC_CU(cudaEventCreate(&e));
        h->ev.push_back(e);
    }
    if (capacity > 0 && !h->g_timed[0]) {
        int r = capture_steps(h, true);
        if (r != RBC_OK) return r;
    }
    h->timing_cap = capacity;
    return RBC_OK;
}

int rbc_kernel_times(rbc_handle *h, double ms[2], int64_t count[2])
{
    if (!h || !ms || !count) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    RBC_CU(cudaStreamSynchronize(h->stream));
    ms[0] = ms[1] = 0.0;
    count[0] = count[1] = 0;
    for (int k = 0; k < h->timing_used; ++k) {
        float a = 0.f, b = 0.f;
        RBC_CU(cudaEventElapsedTime(&a, h->ev[3 * k], h->ev[3 * k + 1]));
        RBC_CU(cudaEventElapsedTime(&b, h->ev[3 * k + 1], h->ev[3 * k + 2]));
        ms[0] += b;
        count[0]++;
        if (h->d.nc > 0) {
            ms[1] += a;
            count[1]++;
        }
    }
    h->timing_used = 0;
    h->timing_cap = 0;
    return RBC_OK;
}

// Re-capture the step graphs (after a change of launch shape), the timed
// ones too if they exist.
static int recapture_steps(rbc_handle *h)
{
    RBC_CU(cudaStreamSynchronize(h->stream));
    int r = capture_steps(h, false);
    if (r == RBC_OK && h->g_timed[0]) r = capture_steps(h, true);
    return r;
}

// ms per coupled step over n steps after n warm-up steps (CUDA events on the
// handle's stream).
static int time_steps(rbc_handle *h, int n, double *ms)
{
    int rc = rbc_step(h, n);
    if (rc != RBC_OK) return rc;
    cudaEvent_t a, b;
    RBC_CU(cudaEventCreate(&a));
    RBC_CU(cudaEventCreate(&b));
    cudaEventRecord(a, h->stream);
    rc = rbc_step(h, n);
    cudaEventRecord(b, h->stream);
    cudaError_t e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return fail(&h->err, RBC_ECUDA, std::string("timing: ") + cudaGetErrorString(e));
    *ms = (double)t / n;
    return rc;
}

int rbc_autotune(rbc_handle *h, int steps_per_trial, rbc_tune_report *out)
{
    if (!h || steps_per_trial < 1) return fail(h ? &h->err : nullptr, RBC_EINVAL, "bad argument");
    rbc_tune_report rep;
    std::memset(&rep, 0, sizeof rep);
    rep.bin_scale = 1.0;
    if (h->timing_used < h->timing_cap) return fail(&h->err, RBC_EINVAL, "kernel timing is active");
    const int st0 = h->d.lb_stages, grid0 = h->d.lb_grid;
    const size_t smem0 = h->d.lb_smem;
    if (h->d.wt_grid != 0 || h->d.gb_grid != 0 || h->split) {
        // the lattice shapes are timed with one block per group of cells and
        // the spread in the per-cell kernel
        h->d.wt_grid = h->d.gb_grid = 0;
        h->split = false;
        const int r = recapture_steps(h);
        if (r != RBC_OK) return r;
    }
    if (grid0 <= 0) {
        int rc = time_steps(h, steps_per_trial, &rep.ms_per_step);
        rep.default_ms_per_step = rep.ms_per_step;
        if (out) *out = rep;
        return rc;
    }
    int rc = time_steps(h, steps_per_trial, &rep.default_ms_per_step);
    if (rc != RBC_OK) return rc;
    int stages[16], ctas[16];
    const int n = lb_shapes(h->d, stages, ctas, 16);
    const bool order0 = h->lb_first;
    double best = rep.default_ms_per_step;
    int best_k = -1;
    for (int k = 0; k < 2 * n; ++k) {
        set_lb_shape(h->d, stages[k % n], ctas[k % n]);
        h->lb_first = k >= n;
        rc = recapture_steps(h);
        double ms = 0.0;
        if (rc == RBC_OK) rc = time_steps(h, steps_per_trial, &ms);
        if (rc != RBC_OK) return rc;
        rep.trials++;
        if (ms < best) {
            best = ms;
            best_k = k;
        }
    }
    if (best_k >= 0) {
        set_lb_shape(h->d, stages[best_k % n], ctas[best_k % n]);
        h->lb_first = best_k >= n;
        rep.stages = stages[best_k % n];
        rep.ctas_per_sm = ctas[best_k % n];
    } else {
        h->d.lb_stages = st0;
        h->d.lb_grid = grid0;
        h->d.lb_smem = smem0;
        h->lb_first = order0;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        rep.stages = st0;
        rep.ctas_per_sm = (grid0 + sms - 1) / sms;
    }
    rep.lattice_first = h->lb_first ? 1 : 0;
    // then, with that shape, the schedule of the cell-side kernels, jointly:
    // the spread in the per-cell kernel or split off it (the side kernels
    // then start beside it), both graph orders, and the grids of the
    // shape-list and Gay-Berne kernels (blocks per SM; 0: one block per
    // group of cells; a bounded grid leaves room on every SM beside each
    // other and beside the spread and the lattice pass)
    if (h->d.nc > 0) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int side[][2] = {{0, 0}, {2, 2}, {3, 2}, {2, 3}, {3, 3}, {4, 2}};
        const bool order1 = h->lb_first;
        bool bsplit = false, border = order1;
        int bw = 0, bg = 0;
        for (int sp = 0; sp < 2; ++sp)
            for (int ord = 0; ord < 2; ++ord)
                for (const auto &c : side) {
                    if (!sp && (ord == 1) == order1 && c[0] == 0 && c[1] == 0) continue;  // timed above
                    h->split = sp == 1;
                    h->lb_first = ord == 1;
                    h->d.wt_grid = c[0] * sms;
                    h->d.gb_grid = c[1] * sms;
                    rc = recapture_steps(h);
                    double ms = 0.0;
                    if (rc == RBC_OK) rc = time_steps(h, steps_per_trial, &ms);
                    if (rc != RBC_OK) return rc;
                    rep.trials++;
                    if (ms < best) {
                        best = ms;
                        bsplit = h->split;
                        border = h->lb_first;
                        bw = c[0];
                        bg = c[1];
                    }
                }
        h->split = bsplit;
        h->lb_first = border;
        h->d.wt_grid = bw * sms;
        h->d.gb_grid = bg * sms;
        rep.split_spread = bsplit ? 1 : 0;
        rep.lattice_first = border ? 1 : 0;
        rep.wt_blocks_per_sm = bw;
        rep.gb_blocks_per_sm = bg;
        // then the particle bins: edges of r_cut x {1, 1.25, 1.5, 2}
        // (coarser grids scan fewer, fuller bins); the arrays hold the finest
        // grid, and a trial that overflows a bin is dropped
        const int dims[3] = {h->d.nx, h->d.ny, h->d.nz};
        const double bin_min = std::sqrt(std::max(h->P.p.rc2, h->P.p.rcw2));
        int nb0[3];
        double bs0[3];
        for (int a = 0; a < 3; ++a) {
            nb0[a] = h->d.nb[a];
            bs0[a] = h->d.bin_size[a];
        }
        double best_scale = 1.0;
        int best_nb[3] = {nb0[0], nb0[1], nb0[2]};
        for (const double scale : {1.25, 1.5, 2.0}) {
            int nbt[3];
            for (int a = 0; a < 3; ++a) nbt[a] = std::max(1, (int)std::floor(dims[a] / (bin_min * scale)));
            if (nbt[0] == best_nb[0] && nbt[1] == best_nb[1] && nbt[2] == best_nb[2]) continue;
            for (int a = 0; a < 3; ++a) {
                h->d.nb[a] = nbt[a];
                h->d.bin_size[a] = (double)dims[a] / nbt[a];
            }
            h->d.nbins = nbt[0] * nbt[1] * nbt[2];
            rc = recapture_steps(h);
            double ms = 0.0;
            if (rc == RBC_OK) rc = time_steps(h, steps_per_trial, &ms);
            if (rc != RBC_OK) return rc;
            rep.trials++;
            int flags[8];
            RBC_CU(cudaMemcpy(flags, h->d.flags, sizeof flags, cudaMemcpyDeviceToHost));
            if (flags[FLAG_OVERFLOW] & (OVF_BIN | OVF_NBR)) {
                flags[FLAG_OVERFLOW] &= ~(OVF_BIN | OVF_NBR);
                RBC_CU(cudaMemcpy(h->d.flags, flags, sizeof flags, cudaMemcpyHostToDevice));
                continue;  // this grid overflowed a bin: not a candidate
            }
            if (ms < best) {
                best = ms;
                best_scale = scale;
                for (int a = 0; a < 3; ++a) best_nb[a] = nbt[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            h->d.nb[a] = best_nb[a];
            h->d.bin_size[a] = best_scale == 1.0 ? bs0[a] : (double)dims[a] / best_nb[a];
        }
        h->d.nbins = best_nb[0] * best_nb[1] * best_nb[2];
        rep.bin_scale = best_scale;
    }
    rep.ms_per_step = best;
    rc = recapture_steps(h);
    if (out) *out = rep;
    return rc;
}

int rbc_wss_accumulate(rbc_handle *h)
{
    if (!h) return fail(nullptr, RBC_EINVAL, "handle is NULL");
    if (h->d.nwss <= 0 || !h->d.S) return fail(&h->err, RBC_EINVAL, "no wall nodes or no stress output");
    launch_wss(h->d, h->stream);
    RBC_CU(cudaGetLastError());
    h->wss_samples++;
    return RBC_OK;
}

// Checkpoint: a header of 16 int64 words, then the populations of the
// current parity, u, sigma (if stored) and the cell state R, q, V, Omega
// (FP64) and the cached-step flags.
namespace {
constexpr int64_t kCkptMagic = 0x3154504b43434252LL;  // "RBCCKPT1"
constexpr int kCkptWords = 16;

size_t ckpt_bytes(const rbc_handle *h)
{
    const Dev &d = h->d;
    const size_t Np = (size_t)d.Np, n = (size_t)d.nc;
    return kCkptWords * 8 + 19 * Np * (size_t)pop_bytes(d.prec) + Np * sizeof(float4) +
           (d.S ? Np * (sizeof(float4) + sizeof(float)) : 0) + n * (3 + 4 + 3 + 3) * sizeof(double) +
           n * sizeof(int);
}

void ckpt_header(const rbc_handle *h, int64_t w[kCkptWords])
{
    const Dev &d = h->d;
    for (int k = 0; k < kCkptWords; ++k) w[k] = 0;
    w[0] = kCkptMagic;
    w[1] = d.nx;
    w[2] = d.ny;
    w[3] = d.nz;
    w[4] = d.nc;
    w[5] = d.prec;
    w[6] = d.compact;
    w[7] = d.Np;
    w[8] = d.S ? 1 : 0;
    w[9] = (int64_t)ckpt_bytes(h);
}
}  // namespace

int rbc_checkpoint_size(const rbc_handle *h, size_t *bytes)
{
    if (!h || !bytes) return fail(nullptr, RBC_EINVAL, "NULL argument");
    *bytes = ckpt_bytes(h);
    return RBC_OK;
}

int rbc_save(rbc_handle *h, void *buf, size_t bytes)
{
    if (!h || !buf) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    if (bytes < ckpt_bytes(h)) return fail(&h->err, RBC_EINVAL, "checkpoint buffer too small");
    const Dev &d = h->d;
    int64_t w[kCkptWords];
    ckpt_header(h, w);
    unsigned long long lb_step = 0, clamps = 0;
    RBC_CU(cudaMemcpyAsync(&lb_step, d.lb_step, sizeof lb_step, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaMemcpyAsync(&clamps, d.clamps, sizeof clamps, cudaMemcpyDeviceToHost, h->stream));
    char *o = static_cast<char *>(buf) + kCkptWords * 8;
    const size_t Np = (size_t)d.Np, n = (size_t)d.nc;
    auto take = [&](const void *src, size_t nb) -> cudaError_t {
        const cudaError_t e = cudaMemcpyAsync(o, src, nb, cudaMemcpyDeviceToHost, h->stream);
        o += nb;
        return e;
    };
    RBC_CU(take(d.pops[h->step & 1], 19 * Np * (size_t)pop_bytes(d.prec)));
    RBC_CU(take(d.U, Np * sizeof(float4)));
    if (d.S) RBC_CU(take(d.S, Np * sizeof(float4)));
    if (d.Syz) RBC_CU(take(d.Syz, Np * sizeof(float)));
    if (n) {
        RBC_CU(take(d.R, 3 * n * sizeof(double)));
        RBC_CU(take(d.q, 4 * n * sizeof(double)));
        RBC_CU(take(d.V, 3 * n * sizeof(double)));
        RBC_CU(take(d.Om, 3 * n * sizeof(double)));
        RBC_CU(take(d.have, n * sizeof(int)));
    }
    RBC_CU(cudaStreamSynchronize(h->stream));
    w[10] = h->step;
    w[11] = (int64_t)lb_step;
    w[12] = (int64_t)clamps;
    std::memcpy(buf, w, sizeof w);
    return check_flags(h);
}

int rbc_load(rbc_handle *h, const void *buf, size_t bytes)
{
    if (!h || !buf) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    int64_t w[kCkptWords], mine[kCkptWords];
    if (bytes < sizeof w) return fail(&h->err, RBC_EINVAL, "checkpoint too short");
    std::memcpy(w, buf, sizeof w);
    ckpt_header(h, mine);
    for (int k = 0; k < 10; ++k)
        if (w[k] != mine[k])
            return fail(&h->err, RBC_EINVAL, "checkpoint of another problem (lattice, cells, storage or layout)");
    if (bytes < ckpt_bytes(h)) return fail(&h->err, RBC_EINVAL, "checkpoint too short");
    Dev &d = h->d;
    RBC_CU(cudaStreamSynchronize(h->stream));
    h->step = w[10];
    const unsigned long long lb_step = (unsigned long long)w[11], clamps = (unsigned long long)w[12];
    const char *o = static_cast<const char *>(buf) + kCkptWords * 8;
    const size_t Np = (size_t)d.Np, n = (size_t)d.nc;
    auto put = [&](void *dst, size_t nb) -> cudaError_t {
        const cudaError_t e = cudaMemcpyAsync(dst, o, nb, cudaMemcpyHostToDevice, h->stream);
        o += nb;
        return e;
    };
    RBC_CU(put(d.pops[h->step & 1], 19 * Np * (size_t)pop_bytes(d.prec)));
    RBC_CU(put(d.U, Np * sizeof(float4)));
    if (d.S) RBC_CU(put(d.S, Np * sizeof(float4)));
    if (d.Syz) RBC_CU(put(d.Syz, Np * sizeof(float)));
    if (n) {
        RBC_CU(put(d.R, 3 * n * sizeof(double)));
        RBC_CU(put(d.q, 4 * n * sizeof(double)));
        RBC_CU(put(d.V, 3 * n * sizeof(double)));
        RBC_CU(put(d.Om, 3 * n * sizeof(double)));
        RBC_CU(put(d.have, n * sizeof(int)));
    }
    RBC_CU(cudaMemcpyAsync(d.lb_step, &lb_step, sizeof lb_step, cudaMemcpyHostToDevice, h->stream));
    RBC_CU(cudaMemcpyAsync(d.clamps, &clamps, sizeof clamps, cudaMemcpyHostToDevice, h->stream));
    // between steps the spread force density is zero; the cell list, the
    // Gay-Berne forces and the shape lists of the restored poses are rebuilt
    // (the shape lists of step k live in buffer k & 1)
    if (d.G) RBC_CU(cudaMemsetAsync(d.G, 0, Np * sizeof(float4), h->stream));
    RBC_CU(cudaMemsetAsync(d.flags, 0, 8 * sizeof(int), h->stream));
    if (n) {
        launch_bin(d, h->P.p, h->stream);
        launch_gb(d, h->P.p, h->stream);
        launch_weights(d, h->P.p, (int)(h->step & 1), h->stream);
    }
    RBC_CU(cudaStreamSynchronize(h->stream));
    RBC_CU(cudaGetLastError());
    return RBC_OK;
}

int rbc_set_wait_limit(rbc_handle *h, int64_t cycles, int starve_batch)
{
    if (!h || cycles < 0 || starve_batch < -1) return fail(h ? &h->err : nullptr, RBC_EINVAL, "bad argument");
    if (h->d.lb_grid <= 0) return fail(&h->err, RBC_EINVAL, "the lattice pass of this solve is not staged");
    h->d.wait_cycles = cycles;
    h->d.starve_batch = starve_batch;
    return recapture_steps(h);
}

int rbc_profile_accumulate(rbc_handle *h, int axis)
{
    if (!h) return fail(nullptr, RBC_EINVAL, "handle is NULL");
    if (axis < 0 || axis > 2) return fail(&h->err, RBC_EINVAL, "axis must be 0, 1 or 2");
    if (h->d.nc <= 0) return fail(&h->err, RBC_EINVAL, "no cells");
    if (axis != h->profile_axis) {
        const int nb = std::max(h->d.nx, std::max(h->d.ny, h->d.nz));
        RBC_CU(cudaMemsetAsync(h->d.profile, 0, sizeof(double) * (size_t)nb, h->stream));
        h->profile_axis = axis;
        h->profile_samples = 0;
    }
    launch_profile(h->d, axis, h->stream);
    RBC_CU(cudaGetLastError());
    h->profile_samples++;
    return RBC_OK;
}

int rbc_profile(rbc_handle *h, double *counts, int nbins, int *axis, int64_t *samples)
{
    if (!h || !counts || !axis || !samples) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    *axis = h->profile_axis;
    *samples = h->profile_samples;
    if (h->profile_axis < 0) {
        for (int k = 0; k < nbins; ++k) counts[k] = 0.0;
        return RBC_OK;
    }
    const int n = h->profile_axis == 0 ? h->d.nx : (h->profile_axis == 1 ? h->d.ny : h->d.nz);
    if (nbins < n) return fail(&h->err, RBC_EINVAL, "nbins is smaller than the box along the axis");
    RBC_CU(cudaMemcpyAsync(counts, h->d.profile, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    for (int k = n; k < nbins; ++k) counts[k] = 0.0;
    return RBC_OK;
}

int rbc_wss(rbc_handle *h, int64_t *node, double *tau, int64_t max, int64_t *n, int64_t *samples)
{
    if (!h || !n || !samples || (max > 0 && (!node || !tau)))
        return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    if (h->d.nwss <= 0 || !h->d.S) return fail(&h->err, RBC_EINVAL, "no wall nodes or no stress output");
    const size_t nw = (size_t)h->d.nwss;
    std::vector<int> idx(nw);
    std::vector<double> acc(3 * nw);
    RBC_CU(cudaMemcpyAsync(idx.data(), h->d.wss_node, nw * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaMemcpyAsync(acc.data(), h->d.wss_acc, 3 * nw * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RBC_CU(cudaStreamSynchronize(h->stream));
    const double inv = h->wss_samples > 0 ? 1.0 / (double)h->wss_samples : 0.0;
    const size_t k = std::min(nw, (size_t)std::max<int64_t>(max, 0));
    for (size_t i = 0; i < k; ++i) {
        node[i] = h->d.compact ? h->wss_dense[i] : idx[i];
        for (int a = 0; a < 3; ++a) tau[3 * i + a] = acc[3 * i + a] * inv;
    }
    *n = (int64_t)nw;
    *samples = h->wss_samples;
    return RBC_OK;
}

int rbc_set_schedule(rbc_handle *h, int split_spread, int lattice_first)
{
    if (!h) return fail(nullptr, RBC_EINVAL, "handle is NULL");
    if (h->timing_used < h->timing_cap) return fail(&h->err, RBC_EINVAL, "kernel timing is active");
    h->split = split_spread != 0 && h->d.nc > 0;
    h->lb_first = lattice_first != 0;
    return recapture_steps(h);
}

int rbc_launches_per_step(const rbc_handle *h)
{
    if (!h) return 0;
    // lattice pass; cells, bin, gb, weights (+ the spread when split); the
    // bin-count clear is a memset node
    return 1 + (h->d.nc > 0 ? (h->split ? 5 : 4) : 0);
}

int rbc_layout(const rbc_handle *h, int *compact, int64_t *entries, int64_t *fluid)
{
    if (!h) return fail(nullptr, RBC_EINVAL, "handle is NULL");
    if (compact) *compact = h->d.compact;
    if (entries) *entries = h->d.compact ? h->d.M : h->d.N;
    if (fluid) *fluid = h->P.nfluid;
    return RBC_OK;
}

int rbc_fluid_nodes(rbc_handle *h, int64_t *nodes, int64_t max, int64_t *count)
{
    if (!h || !count || (max > 0 && !nodes)) return fail(h ? &h->err : nullptr, RBC_EINVAL, "NULL argument");
    const Dev &d = h->d;
    int64_t k = 0;
    auto put = [&](int64_t n) {
        if (k < max) nodes[k] = n;
        ++k;
    };
    if (d.compact) {
        // walk the device's own row table and link words in storage order
        std::vector<int4> rows((size_t)d.ny * d.nz);
        std::vector<uint32_t> links((size_t)d.M);
        RBC_CU(cudaMemcpyAsync(rows.data(), d.rows, rows.size() * sizeof(int4), cudaMemcpyDeviceToHost, h->stream));
        RBC_CU(cudaMemcpyAsync(links.data(), d.links, links.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                               h->stream));
        RBC_CU(cudaStreamSynchronize(h->stream));
        std::vector<std::pair<int64_t, int64_t>> order;  // (entry, node) of the fluid entries
        for (size_t r = 0; r < rows.size(); ++r)
            for (int x = rows[r].y; x < rows[r].z; ++x) {
                const int64_t c = (int64_t)rows[r].x + (x - rows[r].y);
                if (c < 0 || c >= d.M) return fail(&h->err, RBC_EINVAL, "row table outside the storage");
                if (x < d.nx && !(links[(size_t)c] >> 31)) order.emplace_back(c, (int64_t)d.nx * (int64_t)r + x);
            }
        std::sort(order.begin(), order.end());
        for (const auto &e : order) put(e.second);
    } else if (d.links) {
        std::vector<uint32_t> links((size_t)d.N);
        RBC_CU(cudaMemcpyAsync(links.data(), d.links, links.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                               h->stream));
        RBC_CU(cudaStreamSynchronize(h->stream));
        for (int64_t n = 0; n < d.N; ++n)
            if (!(links[(size_t)n] >> 31)) put(n);
    } else {
        for (int64_t n = 0; n < d.N; ++n) put(n);
    }
    *count = k;
    return RBC_OK;
}

void rbc_free(rbc_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->g_pro) cudaGraphExecDestroy(h->g_pro);
    for (int k = 0; k < 2; ++k) {
        if (h->g_step[k]) cudaGraphExecDestroy(h->g_step[k]);
        if (h->g_timed[k]) cudaGraphExecDestroy(h->g_timed[k]);
        if (h->src_timed[k]) cudaGraphDestroy(h->src_timed[k]);
    }
    for (int k = 0; k < 3; ++k)
        if (h->src[k]) cudaGraphDestroy(h->src[k]);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    for (int k = 0; k < 3; ++k)
        if (h->ev_dummy[k]) cudaEventDestroy(h->ev_dummy[k]);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->join2_ev) cudaEventDestroy(h->join2_ev);
    if (h->side2) {
        cudaStreamSynchronize(h->side2);
        cudaStreamDestroy(h->side2);
    }
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char *rbc_last_error(const rbc_handle *h)
{
    if (h) return h->err.c_str();
    return g_thread_err.c_str();
}

}  // extern "C"
