// logm_small_v1.cu -- the one-block-per-matrix kernels in their 128-thread
// configuration for n <= 64 (32 x 32 DMMA tiles, up to 5 blocks per SM), so
// that more small matrices are in flight per SM than with 256-thread blocks.
#define LG_NS lg_v1
#define LG_THREADS 128
#define LG_MAXN 64
#define LG_TILE 32
#define LG_MINBLOCKS 5
#include "logm_small.cu"
