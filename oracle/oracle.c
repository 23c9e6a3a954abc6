/*
 * CPU oracle for Bayer-domain block motion estimation and motion-vector
 * feature propagation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library under paper_2508_05990_b300/) shares no code with it and must
 * never call it.
 *
 * Everything here is written to be read against the paper:
 *   "Efficient Bayer-Domain Video Computer Vision with Fast Motion Estimation
 *    and Learned Perception Residual" (arXiv 2508.05990).
 *
 *   Sec. 2.2 "Definition":  MV = ME(F_R, F_C);  F_C = Warp(F_R, MV) + Res.
 *   Sec. 3.2 "Pyramid Block Structure": block sizes large to small, full
 *            resolution at every level, only the block size changes.
 *   Sec. 3.2 "Parallel Coarse-to-fine Block Matching": three stages (coarse,
 *            intermediate, fine), each narrowing range and step.
 *   Sec. 3.2 "Matching Criterion": SAD; the lowest-SAD candidate wins; the
 *            offset between matched block positions is the MV.
 *   Sec. 4.1 "CUDA Settings": (2R+1)^2 candidates per block per stage, R the
 *            search radius counted in steps; the MV field is h x w.
 *   FME-settings table (Sec. 4.2, commented out in the source): standard
 *            setting blocks [64,32], stages (R,step) = (8,8),(4,4),(2,1).
 *   Sec. 3.3 equation z_C = Warp(z_R, MV) + z_Res: the propagation.
 *
 * Readings where the paper is silent (stated once here, applied below):
 *   - MV sign: the current block at (x, y) matches the reference block at
 *     (x + dx, y + dy).
 *   - A candidate whose displaced block leaves the frame is skipped.
 *   - Partial edge blocks are clipped to the frame; SAD covers in-frame pixels.
 *   - Tie-break: lexicographic minimum of (sad, |dx|+|dy|, dy, dx) on the
 *     absolute MV.
 *   - CFA phase: EVEN mode uses even offsets only (like-coloured samples of the
 *     RGGB mosaic are compared); RAW mode uses every integer offset.
 *   - Propagation: feature cell (fy, fx) takes the MV of the block holding raw
 *     pixel (fy*s, fx*s); the source position is (fy + dy/s, fx + dx/s).
 *     NEAREST rounds dy/s, dx/s half away from zero; BILINEAR weights the
 *     four neighbours in a fixed evaluation order; indices are clamped.
 *
 * Plain loops throughout: no blocking, fusion or reordering of the arithmetic.
 * OpenMP only distributes independent blocks (or feature rows) over threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int16_t dx;
  int16_t dy;
  uint32_t sad;
} omv_t; /* one MV record: 8 bytes */

/* -------------------------------------------------------------------------- */
/* threads                                                                    */
/* -------------------------------------------------------------------------- */

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* -------------------------------------------------------------------------- */
/* motion estimation                                                          */
/* -------------------------------------------------------------------------- */

/* Tie-break order on candidates (reading of Sec. 3.2 "Matching Criterion"):
 * returns 1 when candidate a is preferred over candidate b. */
static int better(uint64_t sad_a, int dx_a, int dy_a, uint64_t sad_b, int dx_b, int dy_b) {
  if (sad_a != sad_b) return sad_a < sad_b;
  int l1a = abs(dx_a) + abs(dy_a), l1b = abs(dx_b) + abs(dy_b);
  if (l1a != l1b) return l1a < l1b;
  if (dy_a != dy_b) return dy_a < dy_b;
  return dx_a < dx_b;
}

/* SAD of the current block at (x0, y0) of size bw x bh against the reference
 * block displaced by (dx, dy) (Sec. 3.2 "Matching Criterion"). */
static uint64_t block_sad(const uint16_t* ref, const uint16_t* cur, int pitch, int x0, int y0,
                          int bw, int bh, int dx, int dy) {
  uint64_t s = 0;
  for (int y = 0; y < bh; ++y) {
    const uint16_t* c = cur + (size_t)(y0 + y) * pitch + x0;
    const uint16_t* r = ref + (size_t)(y0 + y + dy) * pitch + x0 + dx;
    for (int x = 0; x < bw; ++x) {
      int d = (int)c[x] - (int)r[x];
      s += (uint64_t)(d < 0 ? -d : d);
    }
  }
  return s;
}

/* One matching stage for one block (Sec. 3.2 coarse-to-fine; Sec. 4.1):
 * candidates {center + (u*step, v*step) : u, v in [-R, R]}, additionally
 * limited to |dx|, |dy| <= lim.  Invalid candidates are skipped.  Returns the
 * best candidate in *best and adds the scheduled pixel-candidate count
 * (every enumerated candidate x block pixels, valid or not) to *count.
 * Returns 0 when no candidate was valid. */
static int stage_one_block(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                           int x0, int y0, int bw, int bh, int cx, int cy, int R, int step,
                           int lim, omv_t* best, long long* count) {
  int have = 0;
  uint64_t bsad = 0;
  int bdx = 0, bdy = 0;
  for (int v = -R; v <= R; ++v) {
    for (int u = -R; u <= R; ++u) {
      int dx = cx + u * step, dy = cy + v * step;
      *count += (long long)bw * bh;
      if (abs(dx) > lim || abs(dy) > lim) continue;
      if (x0 + dx < 0 || x0 + dx + bw > W || y0 + dy < 0 || y0 + dy + bh > H) continue;
      uint64_t s = block_sad(ref, cur, pitch, x0, y0, bw, bh, dx, dy);
      if (!have || better(s, dx, dy, bsad, bdx, bdy)) {
        have = 1;
        bsad = s;
        bdx = dx;
        bdy = dy;
      }
    }
  }
  if (have) {
    if (bsad > 0xFFFFFFFFull) abort(); /* a uint32 SAD is part of the record */
    best->dx = (int16_t)bdx;
    best->dy = (int16_t)bdy;
    best->sad = (uint32_t)bsad;
  }
  return have;
}

/* One stage over the whole block grid h = ceil(H/B), w = ceil(W/B).
 * center: per-block centre MV (NULL = zero MV).  out: h*w records.
 * Returns the scheduled pixel-candidate count, or -1 if some block had no
 * valid candidate. */
long long oracle_me_stage(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                          int B, int R, int step, int lim, const omv_t* center, omv_t* out) {
  int h = (H + B - 1) / B, w = (W + B - 1) / B;
  long long total = 0;
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total) reduction(| : fail)
  for (int b = 0; b < h * w; ++b) {
    int i = b / w, j = b % w;
    int x0 = j * B, y0 = i * B;
    int bw = (x0 + B <= W) ? B : W - x0;
    int bh = (y0 + B <= H) ? B : H - y0;
    int cx = center ? center[b].dx : 0, cy = center ? center[b].dy : 0;
    long long cnt = 0;
    if (!stage_one_block(ref, cur, W, H, pitch, x0, y0, bw, bh, cx, cy, R, step, lim, &out[b], &cnt))
      fail = 1;
    total += cnt;
  }
  return fail ? -1 : total;
}

/* Exhaustive full search (the definition of block matching, Sec. 2.2): every
 * offset with |dx|, |dy| <= range; EVEN phase mode uses even offsets only. */
long long oracle_me_full(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, int B,
                         int range, int even, omv_t* out) {
  int step = even ? 2 : 1;
  return oracle_me_stage(ref, cur, W, H, pitch, B, range / step, step, range, NULL, out);
}

/* Paper coarse-to-fine block pyramid (Sec. 3.2; FME-settings table).
 * levels[0..nlev-1]: block sizes, large to small.  Each level runs the stages
 * (stageR[k], stageS[k]) in order; each stage is centred on the previous
 * stage's best; level 0 starts at the zero MV; level l > 0 starts at the MV of
 * the parent block of level l-1 (the parent block holds the child's top-left
 * pixel).  In EVEN mode an odd step s becomes s' = s + 1 and R becomes
 * floor(R*s/s'), keeping the reach and the CFA phase.
 * out: field of the last level (h*w for the smallest block size).  Returns the scheduled pixel-candidate count. */
long long oracle_me_c2f(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch,
                        const int* levels, int nlev, const int* stageR, const int* stageS, int nst,
                        int even, omv_t* out) {
  long long total = 0;
  omv_t* prev = NULL;
  int prevB = 0, prev_w = 0;
  for (int l = 0; l < nlev; ++l) {
    int B = levels[l];
    int h = (H + B - 1) / B, w = (W + B - 1) / B;
    omv_t* cur_field = (l == nlev - 1) ? out : (omv_t*)malloc(sizeof(omv_t) * (size_t)h * w);
    /* level start: zero MV, or the parent block's MV */
    for (int b = 0; b < h * w; ++b) {
      int i = b / w, j = b % w;
      if (prev) {
        int pi = (i * B) / prevB, pj = (j * B) / prevB;
        cur_field[b] = prev[pi * prev_w + pj];
      } else {
        cur_field[b].dx = 0;
        cur_field[b].dy = 0;
        cur_field[b].sad = 0;
      }
    }
    omv_t* tmp = (omv_t*)malloc(sizeof(omv_t) * (size_t)h * w);
    for (int k = 0; k < nst; ++k) {
      int R = stageR[k], s = stageS[k];
      if (even && (s & 1)) {
        int s2 = s + 1;
        R = (R * s) / s2;
        s = s2;
      }
      long long c = oracle_me_stage(ref, cur, W, H, pitch, B, R, s, 1 << 30, cur_field, tmp);
      if (c < 0) abort(); /* the centre candidate is always valid */
      total += c;
      memcpy(cur_field, tmp, sizeof(omv_t) * (size_t)h * w);
    }
    free(tmp);
    if (prev) free(prev);
    prev = (l == nlev - 1) ? NULL : cur_field;
    prevB = B;
    prev_w = w;
  }
  return total;
}

/* Learned-seeded search (the refine-around-a-proposal form of the method):
 * per block, conf < thresh -> full search (EVEN, +-range); otherwise the
 * proposal is rounded to the nearest even integer (half away from zero),
 * clamped to [-range, range] and then to the valid displacement interval of
 * the block, and one stage R = 2, step = 2 is searched around it with
 * |dx|, |dy| <= range.  fallback[b] = 1 when block b used the full search. */
long long oracle_me_seeded(const uint16_t* ref, const uint16_t* cur, int W, int H, int pitch, int B,
                           int range, const float* prop_dx, const float* prop_dy, const float* conf,
                           float thresh, omv_t* out, uint8_t* fallback) {
  int h = (H + B - 1) / B, w = (W + B - 1) / B;
  long long total = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total)
  for (int b = 0; b < h * w; ++b) {
    int i = b / w, j = b % w;
    int x0 = j * B, y0 = i * B;
    int bw = (x0 + B <= W) ? B : W - x0;
    int bh = (y0 + B <= H) ? B : H - y0;
    long long cnt = 0;
    if (!(conf[b] >= thresh)) {
      fallback[b] = 1;
      stage_one_block(ref, cur, W, H, pitch, x0, y0, bw, bh, 0, 0, range / 2, 2, range, &out[b], &cnt);
    } else {
      fallback[b] = 0;
      /* proposals beyond +-1024 are first limited to +-1024 (the centre is
       * clamped to +-range <= 510 below anyway); this keeps the float-to-int
       * conversion defined for any input */
      float px = fminf(fmaxf(prop_dx[b], -1024.f), 1024.f);
      float py = fminf(fmaxf(prop_dy[b], -1024.f), 1024.f);
      int cx = 2 * (int)roundf(px * 0.5f);
      int cy = 2 * (int)roundf(py * 0.5f);
      if (cx < -range) cx = -range;
      if (cx > range) cx = range;
      if (cy < -range) cy = -range;
      if (cy > range) cy = range;
      if (cx < -x0) cx = -x0;
      if (cx > W - bw - x0) cx = W - bw - x0;
      if (cy < -y0) cy = -y0;
      if (cy > H - bh - y0) cy = H - bh - y0;
      stage_one_block(ref, cur, W, H, pitch, x0, y0, bw, bh, cx, cy, 2, 2, range, &out[b], &cnt);
    }
    total += cnt;
  }
  return total;
}

/* -------------------------------------------------------------------------- */
/* propagation (Sec. 3.3: z_pred = Warp(z_R, MV))                             */
/* -------------------------------------------------------------------------- */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor(a / b) for b > 0 */
static int floordiv(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

/* a / b rounded half away from zero, b > 0 */
static int rounddiv(int a, int b) {
  if (a >= 0) return (2 * a + b) / (2 * b);
  return -((2 * (-a) + b) / (2 * b));
}

/* element offset of (c, y, x) for NCHW (layout 0) or NHWC (layout 1) */
static size_t fidx(int layout, int C, int Hf, int Wf, int c, int y, int x) {
  if (layout == 0) return ((size_t)c * Hf + y) * Wf + x;
  return ((size_t)y * Wf + x) * C + c;
}

/* interp 0 = NEAREST (a copy), 1 = BILINEAR evaluated in float in the order
 *   out = (1-wy)*((1-wx)*a + wx*b) + wy*((1-wx)*c + wx*d)
 * with every product and sum rounded to float (no fused multiply-add). */
void oracle_propagate_f32(const float* feat, int C, int Hf, int Wf, int layout, int interp,
                          const omv_t* mv, int mv_h, int mv_w, int B, int s, float* out) {
  int cells = B / s;
  (void)mv_h;
#pragma omp parallel for schedule(static)
  for (int fy = 0; fy < Hf; ++fy) {
    for (int fx = 0; fx < Wf; ++fx) {
      const omv_t m = mv[(fy / cells) * mv_w + (fx / cells)];
      if (interp == 0) {
        int sy = clampi(fy + rounddiv(m.dy, s), 0, Hf - 1);
        int sx = clampi(fx + rounddiv(m.dx, s), 0, Wf - 1);
        for (int c = 0; c < C; ++c)
          out[fidx(layout, C, Hf, Wf, c, fy, fx)] = feat[fidx(layout, C, Hf, Wf, c, sy, sx)];
      } else {
        int qy = floordiv(m.dy, s), qx = floordiv(m.dx, s);
        float wy = (float)(m.dy - qy * s) / (float)s;
        float wx = (float)(m.dx - qx * s) / (float)s;
        float owy = 1.0f - wy, owx = 1.0f - wx;
        int y0 = clampi(fy + qy, 0, Hf - 1), y1 = clampi(fy + qy + 1, 0, Hf - 1);
        int x0 = clampi(fx + qx, 0, Wf - 1), x1 = clampi(fx + qx + 1, 0, Wf - 1);
        for (int c = 0; c < C; ++c) {
          float a = feat[fidx(layout, C, Hf, Wf, c, y0, x0)];
          float b = feat[fidx(layout, C, Hf, Wf, c, y0, x1)];
          float cc = feat[fidx(layout, C, Hf, Wf, c, y1, x0)];
          float d = feat[fidx(layout, C, Hf, Wf, c, y1, x1)];
          float t0 = owx * a;
          float t1 = wx * b;
          float top = t0 + t1;
          float t2 = owx * cc;
          float t3 = wx * d;
          float bot = t2 + t3;
          float u0 = owy * top;
          float u1 = wy * bot;
          out[fidx(layout, C, Hf, Wf, c, fy, fx)] = u0 + u1;
        }
      }
    }
  }
}

/* The same bilinear propagation evaluated in double (the precision
 * reference for any floating-point form). */
void oracle_propagate_bilinear_f64(const float* feat, int C, int Hf, int Wf, int layout,
                                   const omv_t* mv, int mv_h, int mv_w, int B, int s, double* out) {
  int cells = B / s;
  (void)mv_h;
#pragma omp parallel for schedule(static)
  for (int fy = 0; fy < Hf; ++fy) {
    for (int fx = 0; fx < Wf; ++fx) {
      const omv_t m = mv[(fy / cells) * mv_w + (fx / cells)];
      double ty = (double)m.dy / s, tx = (double)m.dx / s;
      double yy = fy + ty, xx = fx + tx;
      double fy0 = floor(yy), fx0 = floor(xx);
      double wy = yy - fy0, wx = xx - fx0;
      int y0 = clampi((int)fy0, 0, Hf - 1), y1 = clampi((int)fy0 + 1, 0, Hf - 1);
      int x0 = clampi((int)fx0, 0, Wf - 1), x1 = clampi((int)fx0 + 1, 0, Wf - 1);
      for (int c = 0; c < C; ++c) {
        double a = feat[fidx(layout, C, Hf, Wf, c, y0, x0)];
        double b = feat[fidx(layout, C, Hf, Wf, c, y0, x1)];
        double cc = feat[fidx(layout, C, Hf, Wf, c, y1, x0)];
        double d = feat[fidx(layout, C, Hf, Wf, c, y1, x1)];
        out[fidx(layout, C, Hf, Wf, c, fy, fx)] =
            (1.0 - wy) * ((1.0 - wx) * a + wx * b) + wy * ((1.0 - wx) * cc + wx * d);
      }
    }
  }
}
