// logm_small_v5.cu -- the 64-thread configuration for n <= 32 (32 x 32 DMMA
// tiles) with the execute mode's working matrices in the block's shared
// memory instead of an L2-resident workspace slot (7 x n^2 FP64: 57 KB at
// n = 32, 14 KB at n = 16); the grid holds as many blocks as fit.
#define LG_NS lg_v5
#define LG_THREADS 64
#define LG_MAXN 32
#define LG_TILE 32
#define LG_MINBLOCKS 3
#define LG_SMEM_SLOTS 1
#include "logm_small.cu"
