/*
 * Lens-transport ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of what the GPU path
 * computes, written from the paper (Precomputed Lens Transport Maps,
 * Sec. 3 Eq. 1-7 for the traced operator, Sec. 4.2 for path decomposition
 * and the valid/occluded mask, Sec. 5.1 for the map and the networks).
 * Only the test-suite, the smoke check and the benchmark's CPU baseline may
 * load it.  It shares no source with the CUDA library.
 *
 * Units: millimetres, wavelengths in nanometres at the interface (glass
 * formulas take micrometres).  Surfaces are numbered 1..S as in the paper.
 */
#ifndef LT_ORACLE_H
#define LT_ORACLE_H

#include <stdint.h>

#define OR_MAXS 64
#define OR_MAXG 64

enum { OR_AIR = 0, OR_CAUCHY = 1, OR_SELLMEIER = 2 };
enum { OR_T = 0, OR_R = 1 };

typedef struct {
    int S;                          /* optical surfaces */
    double zv[OR_MAXS + 2];         /* vertex z of surface k (1..S) */
    double c[OR_MAXS + 2];          /* curvature 1/R of surface k, 0 = plane */
    double ap[OR_MAXS + 2];         /* clear aperture radius of surface k */
    int asph[OR_MAXS + 2];          /* surface k is an even asphere (conic and polynomial below) */
    double conic[OR_MAXS + 2];      /* conic constant kappa of surface k */
    double a4[OR_MAXS + 2][4];      /* A4, A6, A8, A10 of surface k */
    int med[OR_MAXS + 2];           /* glass of medium m (0..S), -1 = air; m = k is after surface k */
    int n_glass;
    int gkind[OR_MAXG];
    double gA[OR_MAXG], gB[OR_MAXG];
    double gSB[OR_MAXG][3], gSC[OR_MAXG][3];
    int stop_gap;                   /* stop lies in gap g (between surface g and g+1; 0 = in front of 1), -1 none */
    double z_stop, a_stop;
    double z_image;
} or_lens;

#endif
