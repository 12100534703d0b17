// Pool CTA kernel, rank bucket 8.
#define ISVD_TICK_KB 8
#include "pool_tick_inst.cuh"
