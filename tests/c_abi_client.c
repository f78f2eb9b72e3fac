/* A plain C11 client of the library, using nothing but include/rad.h: it shows
 * that the boundary is usable without Python and that the header compiles as
 * C.  Reads a job from a binary file, accumulates every step from host arrays
 * (the library copies them), reads the three spectra back to host memory and
 * writes them to a second file.
 *
 * Input (native byte order):
 *   int32 n_omega, int32 n_dir, int32 n_steps, int32 ff_kind, int64 n,
 *   double ff_width, double omega[n_omega], double dirs[n_dir][3],
 *   then per step: double t, double dt, double r[3][n], double beta[3][n],
 *   double beta_dot[3][n], double w[n].
 * Output: double coherent, incoherent, total, each [n_dir][n_omega].
 * Exit status 0 on success; otherwise a message on stderr. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "rad.h"

static int read_all(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

static int fail(const char* what, rad_status s) {
  fprintf(stderr, "%s: %s\n", what, rad_status_str(s));
  return 1;
}

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s input output\n", argv[0]);
    return 2;
  }
  FILE* in = fopen(argv[1], "rb");
  if (!in) {
    perror(argv[1]);
    return 2;
  }
  int32_t hdr[4];
  int64_t n = 0;
  double width = 0.0;
  if (!read_all(in, hdr, sizeof(hdr)) || !read_all(in, &n, sizeof(n)) ||
      !read_all(in, &width, sizeof(width)) || hdr[0] < 1 || hdr[1] < 1 || hdr[2] < 0 || n < 0) {
    fprintf(stderr, "bad header\n");
    return 2;
  }
  const int32_t n_omega = hdr[0], n_dir = hdr[1], n_steps = hdr[2];
  const size_t bins = (size_t)n_omega * (size_t)n_dir;
  double* omega = malloc(sizeof(double) * (size_t)n_omega);
  double* dirs = malloc(sizeof(double) * 3 * (size_t)n_dir);
  double* part = malloc(sizeof(double) * 10 * (size_t)(n > 0 ? n : 1));
  double* spec = malloc(sizeof(double) * 3 * bins);
  if (!omega || !dirs || !part || !spec) return 2;
  if (!read_all(in, omega, sizeof(double) * (size_t)n_omega) ||
      !read_all(in, dirs, sizeof(double) * 3 * (size_t)n_dir)) {
    fprintf(stderr, "short grid\n");
    return 2;
  }

  /* An invalid grid is refused with a status, not a crash. */
  rad_ff ff = {hdr[3], 0, width};
  rad_ctx* bad = NULL;
  if (rad_create(omega, 0, dirs, n_dir, ff, RAD_PREC_MIXED, NULL, &bad) != RAD_EINVAL || bad) {
    fprintf(stderr, "rad_create accepted an empty frequency grid\n");
    return 1;
  }

  rad_ctx* ctx = NULL;
  rad_status s = rad_create(omega, n_omega, dirs, n_dir, ff, RAD_PREC_MIXED, NULL, &ctx);
  if (s != RAD_OK) return fail("rad_create", s);
  for (int32_t k = 0; k < n_steps; ++k) {
    double tt[2];
    if (!read_all(in, tt, sizeof(tt)) || !read_all(in, part, sizeof(double) * 10 * (size_t)n)) {
      fprintf(stderr, "short step %d\n", (int)k);
      return 2;
    }
    s = rad_accumulate(ctx, n, part, part + 3 * n, part + 6 * n, part + 9 * n, tt[0], tt[1]);
    if (s != RAD_OK) return fail("rad_accumulate", s);
  }
  fclose(in);
  s = rad_spectrum(ctx, spec, spec + bins, spec + 2 * bins);
  if (s != RAD_OK) return fail("rad_spectrum", s);
  rad_destroy(ctx);

  FILE* out = fopen(argv[2], "wb");
  if (!out || fwrite(spec, sizeof(double), 3 * bins, out) != 3 * bins) {
    perror(argv[2]);
    return 2;
  }
  fclose(out);
  free(omega);
  free(dirs);
  free(part);
  free(spec);
  return 0;
}
