// What the compositing forward reads of the binning workspace when only the
// short tile lists were written (qn_bin_sort_partial): the depth-sorted
// visible Gaussians cut into chunks of BIN_CHUNK, and per chunk a column word
// and a row word per tile column / row and per 32 members (bit j of word w:
// member 32 w + j's rect covers that column / row).  Tile t = (tx, ty) holds
// member m of chunk c iff the bit is set in both words; its list is the
// members of chunk 0, then chunk 1, ..., each in depth order -- the order of
// the stable (tile, depth) sort.
#pragma once

#include <cstddef>
#include <cstdint>

namespace qn {

constexpr int BIN_CHUNK = 256;                          // Gaussians per chunk
constexpr int BIN_CHUNK_WARPS = BIN_CHUNK / 32;         // 32-member words per chunk and tile row / column

struct BinView {
    const uint32_t *masks;   // per chunk: column words [tiles_x][BIN_CHUNK_WARPS], then row words [tiles_y][...]
    const uint32_t *sorted;  // depth-sorted Gaussian indices (visible ones first)
    const uint32_t *n_vis;   // device: the number of visible Gaussians
    const uint32_t *list_max;  // device: the lists of at most this many pairs were written
    const uint32_t *occ;     // [occ_w][tiles]: bit c % 32 of word c / 32 -- chunk c has a member in the tile
    int occ_w;               // ceil(chunks / 32)
    // written by the walk when no list was written (list_max 0), for the
    // adjoint's gather: gbase[c][t] the first list position of chunk c's
    // members in tile t (for the chunks walked), wext[t] the chunk the walk of
    // tile t stopped at (every occupied chunk below it walked)
    uint32_t *gbase;         // [chunks][tiles]
    uint32_t *wext;          // [tiles]
};

// The view of a workspace of qn_bin_sort for n Gaussians on a tiles_x x
// tiles_y grid; QN_OK, or QN_ERR_INVALID_ARG (message set) when the workspace
// is missing, misaligned or too small.
int bin_view(int32_t n, int32_t tiles_x, int32_t tiles_y, void *workspace, size_t workspace_bytes, BinView &v);

}  // namespace qn
