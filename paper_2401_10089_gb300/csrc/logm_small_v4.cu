// logm_small_v4.cu -- configuration 1 (128 threads, n <= 64, 32 x 32 DMMA
// tiles) with seven blocks per SM (registers capped at 72 per thread, a few
// spills). Not a tuning choice: a uniform batch that configuration 1 would
// run in two rounds of 5 blocks per SM but that fits one round of 7 runs
// here (the FP64 pipe is already busy at 5 per SM, so the gain is the
// second, partly empty round).
#define LG_NS lg_v4
#define LG_THREADS 128
#define LG_MAXN 64
#define LG_TILE 32
#define LG_MINBLOCKS 7
#include "logm_small.cu"
