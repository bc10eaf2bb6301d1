// Launch-shape constants of the pair kernels.  Written by the package's
// autotuner (python -m paper_1709_04488_gb300.autotune build), which builds
// variants of the library with -D overrides, times the Sod and Sedov steps
// on the GPU and keeps the fastest value of each constant in turn; a -D
// definition on the nvcc command line still overrides every value here.
#pragma once

// density: staged candidates per chunk, blocks per SM the registers are
// sized for (at several lanes per particle, and at one), list entries per
// lane at one lane per particle
#ifndef SPH_DENS_CH
#define SPH_DENS_CH 64
#endif
#ifndef SPH_DENS_MINB
#define SPH_DENS_MINB 4
#endif
#ifndef SPH_DENS_MINB1
#define SPH_DENS_MINB1 5
#endif
#ifndef SPH_DENS_LCAP1
#define SPH_DENS_LCAP1 96
#endif

// forces: staged candidates per chunk, blocks per SM the registers are sized
// for, table of candidate leaves, list entries per lane and candidates per
// list-room check (each at several lanes per particle, and at one)
#ifndef SPH_FORCE_CH
#define SPH_FORCE_CH 64
#endif
#ifndef SPH_FORCE_MINB
#define SPH_FORCE_MINB 4
#endif
#ifndef SPH_FORCE_MINB1
#define SPH_FORCE_MINB1 5
#endif
#ifndef SPH_FORCE_TAB
#define SPH_FORCE_TAB 64
#endif
#ifndef SPH_FORCE_LC
#define SPH_FORCE_LC 64
#endif
#ifndef SPH_FORCE_SB
#define SPH_FORCE_SB 32
#endif
#ifndef SPH_FORCE_LC1
#define SPH_FORCE_LC1 80
#endif
#ifndef SPH_FORCE_SB1
#define SPH_FORCE_SB1 8
#endif
