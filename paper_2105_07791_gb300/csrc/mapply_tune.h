// Tile rows of the dense 32-column apply tiles (mapply_kernel) by the number
// of rows a node's tiles cover (m_i + m_b going up, m_i coming down):
// bucket q holds the nodes with MAPPLY_BUCKET_EDGES[q - 1] <= rows <
// MAPPLY_BUCKET_EDGES[q].  Written by paper_2105_07791_gb300/autotune.py from
// timed multi applies of the 64-problem Helmholtz batch; NDHSS_MAPPLY_TILES
// ("r0,r1,r2,r3", each 32 or 64) overrides it.
#pragma once
constexpr int MAPPLY_NBUCKET = 4;
constexpr int MAPPLY_BUCKET_EDGES[MAPPLY_NBUCKET - 1] = {48, 96, 192};
// Tuned on a GB300 (16 assignments, median of 10 applies each): 32 rows in
// every bucket 3.93 ms, 64 in every bucket 4.40 ms, slowest 4.74 ms.
constexpr int MAPPLY_TILE_ROWS[MAPPLY_NBUCKET] = {32, 32, 32, 32};
