// Pool CTA kernel, rank bucket 64.
#define ISVD_TICK_KB 64
#include "pool_tick_inst.cuh"
