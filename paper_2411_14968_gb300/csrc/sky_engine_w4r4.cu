// The persistent local-skyline engine with 4 warps per CTA and 4 candidates
// per lane (tiles of 512 candidates); see sky_engine_impl.cuh.
#define SKY_ENGINE_WARPS 4
#define SKY_ENGINE_R 4
#include "sky_engine_impl.cuh"
