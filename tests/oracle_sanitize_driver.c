/*
 * Memory-safety driver for the C oracle: compiled together with
 * oracle/oracle.c under AddressSanitizer and UndefinedBehaviorSanitizer by
 * tests/test_oracle_sanitize.py, it runs every oracle entry point on small
 * ragged frames (blocks clipped at the right and bottom edges, candidates
 * leaving the frame, NEAREST and BILINEAR in both layouts) with buffers sized
 * exactly, so that any read or write past them, any signed overflow or any
 * misaligned access aborts the run.  Exit status 0 means every call finished
 * cleanly; the results themselves are checked by the other oracle tests.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef struct {
  int16_t dx;
  int16_t dy;
  uint32_t sad;
} omv_t;

long long oracle_me_stage(const uint16_t*, const uint16_t*, int, int, int, int, int, int, int, const omv_t*, omv_t*);
long long oracle_me_full(const uint16_t*, const uint16_t*, int, int, int, int, int, int, omv_t*);
long long oracle_me_c2f(const uint16_t*, const uint16_t*, int, int, int, const int*, int, const int*, const int*, int,
                        int, omv_t*);
long long oracle_me_seeded(const uint16_t*, const uint16_t*, int, int, int, int, int, const float*, const float*,
                           const float*, float, omv_t*, uint8_t*);
void oracle_propagate_f32(const float*, int, int, int, int, int, const omv_t*, int, int, int, int, float*);
void oracle_propagate_bilinear_f64(const float*, int, int, int, int, const omv_t*, int, int, int, int, double*);
void oracle_set_threads(int);

static uint32_t rng = 12345u;
static uint32_t next(void) {
  rng = rng * 1664525u + 1013904223u;
  return rng >> 8;
}

static void frames(uint16_t* a, uint16_t* b, int n) {
  for (int i = 0; i < n; ++i) {
    a[i] = (uint16_t)(next() & 4095u);
    b[i] = (uint16_t)(next() & 4095u);
  }
}

int main(void) {
  oracle_set_threads(2);
  const int shapes[][2] = {{40, 24}, {36, 28}, {70, 50}, {16, 16}};
  for (unsigned s = 0; s < sizeof(shapes) / sizeof(shapes[0]); ++s) {
    const int W = shapes[s][0], H = shapes[s][1], pitch = W + (int)(s & 1);
    uint16_t* ref = malloc(sizeof(uint16_t) * (size_t)pitch * H);
    uint16_t* cur = malloc(sizeof(uint16_t) * (size_t)pitch * H);
    frames(ref, cur, pitch * H);
    for (int B = 8; B <= 16; B += 8) {
      const int h = (H + B - 1) / B, w = (W + B - 1) / B;
      omv_t* out = malloc(sizeof(omv_t) * (size_t)h * w);
      omv_t* ctr = malloc(sizeof(omv_t) * (size_t)h * w);
      for (int even = 0; even <= 1; ++even) oracle_me_full(ref, cur, W, H, pitch, B, 12, even, out);
      for (int i = 0; i < h * w; ++i) {
        ctr[i].dx = (int16_t)((int)(next() % 9) - 4);
        ctr[i].dy = (int16_t)((int)(next() % 9) - 4);
        ctr[i].sad = 0;
      }
      oracle_me_stage(ref, cur, W, H, pitch, B, 3, 2, 10, ctr, out);
      float* px = malloc(sizeof(float) * (size_t)h * w);
      float* py = malloc(sizeof(float) * (size_t)h * w);
      float* cf = malloc(sizeof(float) * (size_t)h * w);
      uint8_t* fb = malloc((size_t)h * w);
      for (int i = 0; i < h * w; ++i) {
        px[i] = (float)((int)(next() % 4001) - 2000) * 0.25f;
        py[i] = (float)((int)(next() % 81) - 40) * 0.5f;
        cf[i] = (float)(next() % 100) / 100.0f;
      }
      if (B == 16) oracle_me_seeded(ref, cur, W, H, pitch, B, 12, px, py, cf, 0.5f, out, fb);
      /* propagation of a map at stride 4 by the last field */
      const int st = 4, Hf = (H + st - 1) / st, Wf = (W + st - 1) / st, C = 3;
      if (((Hf * st + B - 1) / B) == h && ((Wf * st + B - 1) / B) == w) {
        float* feat = malloc(sizeof(float) * (size_t)C * Hf * Wf);
        float* fo = malloc(sizeof(float) * (size_t)C * Hf * Wf);
        double* fd = malloc(sizeof(double) * (size_t)C * Hf * Wf);
        for (int i = 0; i < C * Hf * Wf; ++i) feat[i] = (float)(next() % 1000) / 500.0f - 1.0f;
        for (int layout = 0; layout <= 1; ++layout) {
          for (int interp = 0; interp <= 1; ++interp)
            oracle_propagate_f32(feat, C, Hf, Wf, layout, interp, out, h, w, B, st, fo);
          oracle_propagate_bilinear_f64(feat, C, Hf, Wf, layout, out, h, w, B, st, fd);
        }
        free(feat);
        free(fo);
        free(fd);
      }
      free(px);
      free(py);
      free(cf);
      free(fb);
      free(out);
      free(ctr);
    }
    /* coarse-to-fine: levels 16, 8; stages (2,4), (2,2), (1,1) */
    const int levels[2] = {16, 8}, R[3] = {2, 2, 1}, S[3] = {4, 2, 1};
    omv_t* out = malloc(sizeof(omv_t) * (size_t)((H + 7) / 8) * ((W + 7) / 8));
    for (int even = 0; even <= 1; ++even) oracle_me_c2f(ref, cur, W, H, pitch, levels, 2, R, S, 3, even, out);
    free(out);
    free(ref);
    free(cur);
  }
  puts("sanitized oracle runs: ok");
  return 0;
}
