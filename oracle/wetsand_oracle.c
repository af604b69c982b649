/*
 * CPU oracle for the WETSAND alignment hot path: DTW with its optimal path
 * (Eq. 1, Eq. 5 at gamma = 0, Definition "Alignment path"), the similarity
 * score (Eq. 8), one DBA iteration, and Soft-DTW with its gradient (Eqs. 3-7).
 *
 * TEST INFRASTRUCTURE ONLY.  It is plain, slow, obviously-correct C, built by
 * oracle/__init__.py with gcc (-O2 -ffp-contract=off so that every fused
 * multiply-add is the explicit one written here), and it shares no source,
 * header, table or helper with the CUDA library.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Two instantiations of one body: *_f64 (double: the reference precision)
 * and *_f32 (float: the FP32 mirror used where a float comparison decides an
 * integer, i.e. the warping path and everything derived from it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REAL double
#define FMA(a, b, c) fma((a), (b), (c))
#define EXP(x) exp(x)
#define LOG(x) log(x)
#define SQRT(x) sqrt(x)
#define SFX(name) name##_f64
#include "oracle_body.h"
#undef REAL
#undef FMA
#undef EXP
#undef LOG
#undef SQRT
#undef SFX

#define REAL float
#define FMA(a, b, c) fmaf((a), (b), (c))
#define EXP(x) expf(x)
#define LOG(x) logf(x)
#define SQRT(x) sqrtf(x)
#define SFX(name) name##_f32
#include "oracle_body.h"
#undef REAL
#undef FMA
#undef EXP
#undef LOG
#undef SQRT
#undef SFX

int orc_abi_version(void) { return 2; }
