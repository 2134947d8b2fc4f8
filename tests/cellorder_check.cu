// Host-side check of the library's cell numbering (md_internal.cuh) for the
// tile edge it was compiled with (MD_CELL_TILE): on boxes with every residue
// of nc modulo the tile edge, cell_id is a bijection from the nc^3 cells
// into [0, tiles * T^3), cell_coords inverts it, cell_id_z steps along z from
// the column's id, the T^3 cells of a tile are consecutive ids in (x, y, z)
// order, and consecutive tiles follow (tx, ty, tz) with tz fastest.  Prints
// one line and exits non-zero on a mismatch.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../paper_2009_07400_gb300/csrc/md_internal.cuh"

using namespace mdk;

int main()
{
    long bad = 0, cells = 0;
    const int sizes[][3] = {{2, 2, 2}, {3, 3, 3}, {4, 5, 6}, {7, 9, 8}, {5, 3, 11}, {38, 38, 38}};
    for (const auto &nc : sizes) {
        Rep R{};
        for (int d = 0; d < 3; d++) {
            R.nc[d] = nc[d];
            R.nt[d] = (nc[d] + kTile - 1) / kTile;
        }
        R.cell_off = 1000;   // a replica that is not the first
        const int64_t nids = (int64_t)R.nt[0] * R.nt[1] * R.nt[2] * kTile3;
        std::vector<int> seen((size_t)nids, 0);
        for (int cx = 0; cx < nc[0]; cx++)
            for (int cy = 0; cy < nc[1]; cy++) {
                const int32_t col = (int32_t)cell_id(R, cx, cy, 0);
                for (int cz = 0; cz < nc[2]; cz++) {
                    cells++;
                    const int64_t id = cell_id(R, cx, cy, cz);
                    if (id < R.cell_off || id >= R.cell_off + nids || seen[(size_t)(id - R.cell_off)]++) bad++;
                    int x, y, z;
                    cell_coords(R, id, x, y, z);
                    if (x != cx || y != cy || z != cz) bad++;
                    if (cell_id_z(col, cz) != id) bad++;
                    // tile-major order with the tile's cells consecutive
                    const int64_t tile = ((int64_t)(cx / kTile) * R.nt[1] + cy / kTile) * R.nt[2] + cz / kTile;
                    const int64_t local = ((int64_t)(cx % kTile) * kTile + cy % kTile) * kTile + cz % kTile;
                    if (id - R.cell_off != tile * kTile3 + local) bad++;
                }
            }
    }
    if (bad) {
        std::printf("FAIL: %ld mismatches over %ld cells (tile edge %d)\n", bad, cells, kTile);
        return 1;
    }
    std::printf("ok: %ld cells, tile edge %d\n", cells, kTile);
    return 0;
}
