// Pool CTA kernel, rank bucket 32.
#define ISVD_TICK_KB 32
#include "pool_tick_inst.cuh"
