/*
 * SBP 4-2 first derivative and stencil classes shared by the 2D and 3D oracle files.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle; see orc2d.c).
 */
#ifndef ORC_SBP_H
#define ORC_SBP_H
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------------------- */
/* SBP 4-2 operator (Sec. 2.1; App. C.1 "SBP 4-2").  Interior: fourth-order central
 * difference.  Boundary: the four closure rows of the diagonal-norm operator whose norm is
 * H = diag(17/48, 59/48, 43/48, 49/48, 1, ...).  The right end is the mirror image with the
 * sign flipped (D is antisymmetric about the centre of a segment).                        */
static const double ORC_D_INT[5] = {1.0 / 12.0, -2.0 / 3.0, 0.0, 2.0 / 3.0, -1.0 / 12.0};
static const double ORC_D_BND[4][6] = {
    {-24.0 / 17.0, 59.0 / 34.0, -4.0 / 17.0, -3.0 / 34.0, 0.0, 0.0},
    {-1.0 / 2.0, 0.0, 1.0 / 2.0, 0.0, 0.0, 0.0},
    {4.0 / 43.0, -59.0 / 86.0, 0.0, 59.0 / 86.0, -4.0 / 43.0, 0.0},
    {3.0 / 98.0, 0.0, -59.0 / 98.0, 0.0, 32.0 / 49.0, -4.0 / 49.0}};
/* p0 of eq. (int): the (1,1) entry of the norm H with unit index spacing. */
#define ORC_P0 (17.0 / 48.0)

/* Stencil classes, one per point and direction.                                           */
#define CL_INTERIOR 0  /* 5-point central row                                           */
#define CL_LEFT0 1     /* CL_LEFT0 + r : closure row r at the low end of a segment       */
#define CL_RIGHT0 5    /* CL_RIGHT0 + r: closure row r counted from the high end           */
#define CL_HOLE 15     /* inactive point                                                   */

/* Value of a line at index k, which may lie outside [0, n) on a periodic line; a wrap adds
 * `shift` per period (used for coordinates of periodic Cartesian meshes).                  */
static double line_at(const double *f, long stride, int n, int k, double shift) {
  int w = 0;
  while (k < 0) { k += n; w -= 1; }
  while (k >= n) { k -= n; w += 1; }
  return f[(long)k * stride] + (double)w * shift;
}

/* First derivative along one line at index i, using the point's stencil class. */
static double orc_d1(const double *f, long stride, int n, int i, int cls, double shift) {
  double s = 0.0;
  if (cls == CL_INTERIOR) {
    for (int o = -2; o <= 2; ++o) s += ORC_D_INT[o + 2] * line_at(f, stride, n, i + o, shift);
  } else if (cls >= CL_LEFT0 && cls < CL_LEFT0 + 4) {
    int r = cls - CL_LEFT0;
    for (int c = 0; c < 6; ++c) s += ORC_D_BND[r][c] * line_at(f, stride, n, i - r + c, shift);
  } else if (cls >= CL_RIGHT0 && cls < CL_RIGHT0 + 4) {
    int r = cls - CL_RIGHT0;
    for (int c = 0; c < 6; ++c) s -= ORC_D_BND[r][c] * line_at(f, stride, n, i + r - c, shift);
  }
  return s;
}

/* ---------------------------------------------------------------------------------------- */
/* Stencil classes from the active mask (Sec. 2.2 hole cutting; reading: every maximal run of
 * active points along a line is one SBP segment with closures at both ends; a run shorter
 * than 8 points is made inactive, repeated until no such run remains).                     */
static int classify_line(signed char *act, int n, long stride, int per, signed char *cls, long cstride,
                         int *too_short) {
  int nact = 0;
  for (int k = 0; k < n; ++k) nact += act[(long)k * stride] ? 1 : 0;
  for (int k = 0; k < n; ++k) cls[(long)k * cstride] = CL_HOLE;
  if (nact == 0) return 0;
  if (per && nact == n) {
    for (int k = 0; k < n; ++k) cls[(long)k * cstride] = CL_INTERIOR;
    return 0;
  }
  for (int k = 0; k < n; ++k) {
    int prev = per ? (k + n - 1) % n : k - 1;
    int starts = act[(long)k * stride] && (prev < 0 || !act[(long)prev * stride]);
    if (!starts) continue;
    int len = 0;
    while (len < n) {
      int kk = per ? (k + len) % n : k + len;
      if (kk >= n || !act[(long)kk * stride]) break;
      ++len;
    }
    for (int t = 0; t < len; ++t) {
      int kk = per ? (k + t) % n : k + t;
      int c;
      if (t < 4) c = CL_LEFT0 + t;
      else if (t >= len - 4) c = CL_RIGHT0 + (len - 1 - t);
      else c = CL_INTERIOR;
      cls[(long)kk * cstride] = (signed char)c;
    }
    if (len < 8) {
      *too_short = 1;
      for (int t = 0; t < len; ++t) {
        int kk = per ? (k + t) % n : k + t;
        act[(long)kk * stride] = 0;
      }
    }
  }
  return 0;
}

#endif /* ORC_SBP_H */
