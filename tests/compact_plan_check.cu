// Host-side check of the compact lattice pass's batch table (no GPU): the
// set-up's build_compact is compiled in from the library source and run on a
// solid mask read from a file.  Checked for every batch and segment:
//   - every fluid node lies in exactly one segment's range [c0, c1];
//   - windows contain their range widened by one node (or are the whole row
//     when the row wraps along x) and start and end on whole 32-byte sectors;
//   - the segments' windows lie side by side in the stage planes (offsets),
//     fill at most one stage, and a batch holds 1..kMaxSegs segments;
//   - every copy descriptor lies inside its window, starts on a sector in
//     both the source row and the stage, and the batch's byte count equals
//     the sum of its copies (the mbarrier's transaction count).
// Usage: compact_plan_check mask nx ny nz bytes_per_population cells
// Prints one summary line; the exit status is the number of violations
// (capped at 100), or 101 when build_compact rejects the lattice.
#include "../paper_1107_4889_gb300/csrc/api.cu"

#include <cstdio>
#include <fstream>

int main(int argc, char **argv)
{
    if (argc != 7) return 102;
    const int nx = atoi(argv[2]), ny = atoi(argv[3]), nz = atoi(argv[4]);
    const int esz = atoi(argv[5]), cells = atoi(argv[6]);
    std::vector<uint8_t> solid((size_t)nx * ny * nz);
    std::ifstream f(argv[1], std::ios::binary);
    f.read(reinterpret_cast<char *>(solid.data()), (std::streamsize)solid.size());
    if (!f) return 102;
    Problem P;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    if (!build_compact(P, solid.data(), esz, cells != 0)) {
        printf("rejected\n");
        return 101;
    }
    const int node_bytes = 19 * esz + (cells ? 16 : 0) + 4, A = 32 / esz;
    std::vector<uint8_t> cover(solid.size(), 0);
    long long entries = 0, segs = 0;
    int bad = 0, most = 0;
    auto fail = [&](const char *what, long long a, long long b) {
        if (bad < 10) printf("violation: %s (%lld, %lld)\n", what, a, b);
        ++bad;
    };
    for (size_t bi = 0; bi < P.batches.size(); ++bi) {
        const int4 bd = P.batches[bi];
        const int nb = bd.y & 0xFF, total = (int)((uint32_t)bd.y >> 8);
        if (nb < 1 || nb > rbc::kMaxSegs) fail("segments per batch", (long long)bi, nb);
        if ((long long)total * node_bytes > P.stage_bytes) fail("stage overflow", (long long)bi, total);
        most = std::max(most, total);
        long long bytes = 0;
        int off = 0;
        for (int b = 0; b < nb; ++b) {
            const int2 *pd = &P.pool[(size_t)bd.x + (size_t)rbc::kSegDescs * b];
            const int y = pd[9].x, z = pd[9].y;
            const int c0 = pd[10].x & 0xFFFF, c1 = (int)((uint32_t)pd[10].x >> 16);
            const int X0 = pd[10].y & 0xFFFF, W = (int)((uint32_t)pd[10].y >> 16);
            if (y < 0 || y >= ny || z < 0 || z >= nz || c0 > c1 || c1 >= nx) fail("segment position", y, z);
            if (pd[11].x != off) fail("plane offset", pd[11].x, off);
            if (X0 % A || W % A) fail("window not on sectors", X0, W);
            const bool wraps = c0 == 0 || c1 == nx - 1;
            if (wraps ? (X0 != 0 || W < nx) : (X0 > c0 - 1 || X0 + W < c1 + 2)) fail("window", c0, c1);
            for (int x = c0; x <= c1 && x < nx; ++x) {
                const size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
                if (solid[n]) continue;
                if (cover[n]) fail("node in two segments", x, y);
                cover[n] = 1;
            }
            for (int u = 0; u < 9; ++u) {
                const int cnt = (int)((uint32_t)pd[u].y >> 16), at = pd[u].y & 0xFFFF;
                if (cnt == 0) continue;
                if (at + cnt > W) fail("copy outside the window", at, cnt);
                if ((off + at) % A || pd[u].x % A || cnt % A) fail("copy not on sectors", off + at, cnt);
                const int dy = u % 3 - 1, dz = u / 3 - 1;
                const int planes = (dy == 0 || dz == 0) ? 3 : 1;
                bytes += (long long)cnt * (esz * planes + (u == 4 ? (cells ? 16 : 0) + 4 : 0));
            }
            off += W;
            ++segs;
        }
        if (off != total) fail("entries of the batch", off, total);
        if (bytes != bd.z) fail("transaction bytes", bytes, bd.z);
        entries += total;
    }
    long long fluid = 0;
    for (size_t n = 0; n < solid.size(); ++n)
        if (!solid[n]) {
            ++fluid;
            if (!cover[n]) fail("fluid node in no segment", (long long)n, 0);
        }
    const double fill = P.batches.empty() ? 0.0 : (double)entries / ((double)P.batches.size() * most);
    printf("batches %zu segments %lld fluid %lld entries %lld stage_bytes %d fill %.3f violations %d\n",
           P.batches.size(), segs, fluid, entries, P.stage_bytes, fill, bad);
    return std::min(bad, 100);
}
