// logm_small_v3.cu -- the one-block-per-matrix kernels in a 256-thread
// configuration for n <= 256 with three blocks per SM (registers capped at
// 85 per thread; 3 x 75 KB of shared memory), one more matrix in flight per
// SM than configuration 0 at the cost of a few register spills.
#define LG_NS lg_v3
#define LG_THREADS 256
#define LG_MAXN 256
#define LG_TILE 64
#define LG_MINBLOCKS 3
#include "logm_small.cu"
