// The persistent local-skyline engine with 8 warps per CTA and 4 candidates
// per lane (tiles of 1024 candidates); see sky_engine_impl.cuh.
#define SKY_ENGINE_WARPS 8
#define SKY_ENGINE_R 4
#include "sky_engine_impl.cuh"
