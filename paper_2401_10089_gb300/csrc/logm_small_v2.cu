// logm_small_v2.cu -- the one-block-per-matrix kernels in their 64-thread
// configuration for n <= 32 (32 x 32 DMMA tiles, up to 8 blocks per SM).
#define LG_NS lg_v2
#define LG_THREADS 64
#define LG_MAXN 32
#define LG_TILE 32
#define LG_MINBLOCKS 8
#include "logm_small.cu"
