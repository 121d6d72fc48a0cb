// noalloc.cu -- candidate-partner lists of a set of cells without any device
// allocation and without caller-provided scratch.
//
// rbc_neighbors_noalloc builds the same lists as the cell list of the time
// step (rbc_neighbors): bin the cells, scan the 27 surrounding bins, keep the
// partners j != i with |R_i - R_j|^2 < r_cut^2 (minimum image along periodic
// axes, FP64, no fused multiply-add) sorted by index.  Its scratch -- bin
// counts, bin slots and an overflow flag -- lives in one file-scope static
// device array, so a caller that cannot call cudaMalloc (for instance code
// running where the device memory is fully committed to other buffers, or a
// library embedded in a host that forbids allocation outside its own pool)
// only passes its own input and output buffers.
//
// The array is RBC_NOALLOC_SCRATCH_INTS ints (4 MiB) and stays resident on
// every device that loads this library, until the process exits.  Every call
// shares it: calls that overlap on the GPU (on different streams, or from
// different threads) race on it and must be serialised by the caller.  Each
// call looks up the array's device address with cudaGetSymbolAddress while
// the caller's device is current (a host-side name of a __device__ array is
// not a device address), so the address stays right after the context is
// torn down and re-created.  A call copies the overflow flag back and
// synchronises its stream, so it must never be made on a stream that is
// being captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "../../include/rbc.h"

namespace rbc {
void set_thread_error(const std::string &msg);  // api.cu: rbc_last_error(NULL)
}

namespace {

constexpr int kBinCap = 32;    // cells per bin
constexpr int kWarps = 4;      // cells per CTA of the list kernel
constexpr int kMaxList = 128;  // partners kept per cell

// [0] overflow flag, [1 .. nbins] bin counts, then nbins * kBinCap slots
static __device__ __align__(256) int g_scratch[RBC_NOALLOC_SCRATCH_INTS];

int fail(int code, const std::string &msg)
{
    rbc::set_thread_error(msg);
    return code;
}

__device__ __forceinline__ void min_image(double d[3], const int per[3], const double L[3])
{
    for (int a = 0; a < 3; ++a) {
        if (!per[a]) continue;
        if (d[a] > 0.5 * L[a])
            d[a] = __dsub_rn(d[a], L[a]);
        else if (d[a] < -0.5 * L[a])
            d[a] = __dadd_rn(d[a], L[a]);
    }
}

struct Grid {
    int nb[3], per[3];
    double bs[3], L[3], rc2;
};

__device__ __forceinline__ int bin_of(const double *R, const Grid &g)
{
    int b[3];
    for (int a = 0; a < 3; ++a) {
        const int k = (int)floor(R[a] / g.bs[a]);
        b[a] = k < 0 ? 0 : (k >= g.nb[a] ? g.nb[a] - 1 : k);
    }
    return b[0] + g.nb[0] * (b[1] + g.nb[1] * b[2]);
}

__global__ void k_bin_static(int *scratch, const double *__restrict__ pos, int n, Grid g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nbins = g.nb[0] * g.nb[1] * g.nb[2];
    const int bin = bin_of(&pos[3 * i], g);
    const int slot = atomicAdd(&scratch[1 + bin], 1);
    if (slot < kBinCap)
        scratch[1 + nbins + bin * kBinCap + slot] = i;
    else
        atomicOr(&scratch[0], 1);
}

__device__ __forceinline__ void bin_range(int b, int nb, int per, int &lo, int &hi)
{
    if (per) {
        lo = nb >= 3 ? -1 : 0;
        hi = nb >= 2 ? 1 : 0;
    } else {
        lo = b > 0 ? -1 : 0;
        hi = b < nb - 1 ? 1 : 0;
    }
}

__device__ __forceinline__ int wrap_bin(int b, int nb) { return b < 0 ? b + nb : (b >= nb ? b - nb : b); }

// one warp per cell: ballot-compacted candidates, then a rank sort by index
__global__ void __launch_bounds__(32 * kWarps)
k_lists_static(const int *scratch, int *flag, const double *__restrict__ pos, int n, Grid g,
               int *__restrict__ counts, int *__restrict__ lists, int max_per_cell)
{
    __shared__ int s_cand[kWarps][kMaxList];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.x * kWarps + wid;
    if (i >= n) return;
    const int nbins = g.nb[0] * g.nb[1] * g.nb[2];
    const int *count = scratch + 1, *slots = scratch + 1 + nbins;
    const double Ri[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    const int bin = bin_of(Ri, g);
    const int b[3] = {bin % g.nb[0], (bin / g.nb[0]) % g.nb[1], bin / (g.nb[0] * g.nb[1])};
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) bin_range(b[a], g.nb[a], g.per[a], lo[a], hi[a]);
    int cnt = 0;
    for (int oz = lo[2]; oz <= hi[2]; ++oz)
        for (int oy = lo[1]; oy <= hi[1]; ++oy)
            for (int ox = lo[0]; ox <= hi[0]; ++ox) {
                const int bb = wrap_bin(b[0] + ox, g.nb[0]) +
                               g.nb[0] * (wrap_bin(b[1] + oy, g.nb[1]) + g.nb[1] * wrap_bin(b[2] + oz, g.nb[2]));
                const int c = min(count[bb], kBinCap);
                const int k = lane;
                bool pass = false;
                int j = -1;
                if (k < c) {
                    j = slots[bb * kBinCap + k];
                    if (j != i) {
                        double d[3] = {__dsub_rn(Ri[0], pos[3 * j]), __dsub_rn(Ri[1], pos[3 * j + 1]),
                                       __dsub_rn(Ri[2], pos[3 * j + 2])};
                        min_image(d, g.per, g.L);
                        const double r2 =
                            __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
                        pass = r2 < g.rc2;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, pass);
                const int p = cnt + __popc(m & ((1u << lane) - 1u));
                if (pass && p < kMaxList) s_cand[wid][p] = j;
                cnt += __popc(m);
            }
    if (cnt > max_per_cell) {
        if (lane == 0) atomicOr(flag, 2);
        cnt = max_per_cell;
    }
    __syncwarp();
    for (int e = lane; e < cnt; e += 32) {
        const int v = s_cand[wid][e];
        int r = 0;
        for (int f = 0; f < cnt; ++f) r += s_cand[wid][f] < v;
        lists[(long long)i * max_per_cell + r] = v;
    }
    if (lane == 0) counts[i] = cnt;
}

}  // namespace

extern "C" int rbc_neighbors_noalloc(const double *pos, int n, int nx, int ny, int nz, const int periodic[3],
                                     double r_cut, int *counts, int *lists, int max_per_cell, void *stream)
{
    if (n < 0 || nx < 1 || ny < 1 || nz < 1 || !periodic || !(r_cut > 0.0))
        return fail(RBC_EINVAL, "bad argument");
    if (max_per_cell < 1 || max_per_cell > kMaxList) return fail(RBC_EINVAL, "max_per_cell must be 1..128");
    if (n > 0 && (!pos || !counts || !lists)) return fail(RBC_EINVAL, "NULL buffer");
    Grid g;
    const int dims[3] = {nx, ny, nz};
    const std::string too_big = "the cell-list grid of this box exceeds the static scratch (" +
                                std::to_string(RBC_NOALLOC_SCRATCH_INTS) + " ints)";
    // Bins per axis, checked in floating point before any integer cast: a
    // tiny r_cut would overflow the int, and the product of three large
    // axes the 64-bit count.  Each axis stays below the scratch size
    // (2^20), so the product of three fits 64 bits.
    long long nbins = 1;
    for (int a = 0; a < 3; ++a) {
        g.per[a] = periodic[a] ? 1 : 0;
        if (g.per[a] && 2.0 * r_cut >= dims[a]) return fail(RBC_EINVAL, "r_cut must be below half the box");
        const double per_axis = std::floor(dims[a] / r_cut);
        if (!(per_axis < (double)RBC_NOALLOC_SCRATCH_INTS)) return fail(RBC_EINVAL, too_big);
        g.nb[a] = std::max(1, (int)per_axis);
        g.bs[a] = (double)dims[a] / g.nb[a];
        g.L[a] = dims[a];
        nbins *= g.nb[a];
        if (1 + nbins * (1 + kBinCap) > RBC_NOALLOC_SCRATCH_INTS) return fail(RBC_EINVAL, too_big);
    }
    g.rc2 = r_cut * r_cut;
    // the device address of the static array in the current context
    void *addr = nullptr;
    const cudaError_t ea = cudaGetSymbolAddress(&addr, g_scratch);
    if (ea != cudaSuccess) return fail(RBC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ea));
    int *scratch = static_cast<int *>(addr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the flag and the bin counts must start at zero; slots are written before read
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * (size_t)(1 + nbins), s);
    if (e != cudaSuccess) return fail(RBC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if (n > 0) {
        k_bin_static<<<(n + 127) / 128, 128, 0, s>>>(scratch, pos, n, g);
        k_lists_static<<<(n + kWarps - 1) / kWarps, 32 * kWarps, 0, s>>>(scratch, scratch, pos, n, g, counts, lists,
                                                                         max_per_cell);
    }
    int flag = 0;
    e = cudaMemcpyAsync(&flag, scratch, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(RBC_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    if (flag & 1) return fail(RBC_ENOMEM, "more than 32 cells in a cell-list bin");
    if (flag & 2) return fail(RBC_ENOMEM, "a partner list is longer than max_per_cell");
    return RBC_OK;
}
