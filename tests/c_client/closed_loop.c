/* A plain C client of libmpmi (no Python, no torch): the balance bot's fit and
 * ticks through the C ABI alone.
 *
 *   closed_loop fit   <inputs>            host fit only (no device): prints K
 *   closed_loop ticks <inputs> <device>   fit, safety set, session, and one host
 *                                         tick per (x_t, u_h) record: prints the
 *                                         result of each
 *
 * <inputs> is a binary file of little-endian records written by the test:
 *   int64 m; double x[m*4], u[m], x_next[m*4];
 *   int32 n_samples, horizon; uint64 seed; int32 n_ticks;
 *   then n_ticks times: double x_t[4], u_h.
 * Output lines are "K i j value" or "tick t index status n_safe ttv u_r cost
 * executed" with %.17g doubles and the cost as the float's bits, so a caller
 * can compare them exactly.  Exit status 0 on success, 1 on a usage or file
 * error, 2 on a library error (its message goes to stderr). */
#include <inttypes.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mpmi.h"

static int check(int rc, const char* what) {
  if (rc != MPMI_OK) fprintf(stderr, "%s: %d %s\n", what, rc, mpmi_last_error());
  return rc;
}

static int read_exact(FILE* f, void* p, size_t bytes) {
  return fread(p, 1, bytes, f) == bytes ? 0 : -1;
}

int main(int argc, char** argv) {
  if (argc < 3 || (strcmp(argv[1], "fit") != 0 && strcmp(argv[1], "ticks") != 0)) {
    fprintf(stderr, "usage: %s fit|ticks <inputs> [device]\n", argv[0]);
    return 1;
  }
  FILE* f = fopen(argv[2], "rb");
  if (!f) {
    perror(argv[2]);
    return 1;
  }
  int64_t m = 0;
  if (read_exact(f, &m, sizeof m) || m < 1 || m > 10000000) {
    fprintf(stderr, "bad transition count\n");
    return 1;
  }
  double* x = malloc(sizeof(double) * 4 * m);
  double* u = malloc(sizeof(double) * m);
  double* xn = malloc(sizeof(double) * 4 * m);
  if (!x || !u || !xn || read_exact(f, x, sizeof(double) * 4 * m) ||
      read_exact(f, u, sizeof(double) * m) || read_exact(f, xn, sizeof(double) * 4 * m)) {
    fprintf(stderr, "short transition data\n");
    return 1;
  }
  const mpmi_basis_desc bot = {MPMI_BASIS_BALANCE_BOT, 4, 1};
  int status = 0;

  if (strcmp(argv[1], "fit") == 0) {
    double K[12 * 12], residual = 0.0;
    if (check(mpmi_fit_operator(&bot, x, u, xn, m, K, &residual), "fit_operator")) return 2;
    for (int i = 0; i < 12; ++i)
      for (int j = 0; j < 12; ++j) printf("K %d %d %.17g\n", i, j, K[12 * i + j]);
    printf("residual %.17g\n", residual);
    return 0;
  }

  int32_t n_samples = 0, horizon = 0, n_ticks = 0;
  uint64_t seed = 0;
  if (read_exact(f, &n_samples, 4) || read_exact(f, &horizon, 4) || read_exact(f, &seed, 8) ||
      read_exact(f, &n_ticks, 4) || n_ticks < 0) {
    fprintf(stderr, "short tick header\n");
    return 1;
  }
  const int device = argc > 3 ? atoi(argv[3]) : 0;
  mpmi_ctx* ctx = NULL;
  mpmi_model* model = NULL;
  mpmi_session* sess = NULL;
  if (check(mpmi_create(device, 0, &ctx), "create")) return 2;
  double residual = 0.0;
  if (check(mpmi_fit_model(ctx, &bot, x, u, xn, m, &model, &residual), "fit_model")) {
    status = 2;
    goto done;
  }
  mpmi_safety_spec spec;
  memset(&spec, 0, sizeof spec);
  for (int j = 0; j < MPMI_MAX_NX; ++j) {
    spec.state_lo[j] = -INFINITY;
    spec.state_hi[j] = INFINITY;
  }
  spec.state_lo[0] = -0.5; /* |theta| < 0.5 rad */
  spec.state_hi[0] = 0.5;
  spec.state_lo[2] = -2.0; /* |x| < 2 m */
  spec.state_hi[2] = 2.0;
  if (check(mpmi_set_safety_set(model, &spec), "set_safety_set")) {
    status = 2;
    goto done;
  }
  mpmi_session_config cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.n_samples = n_samples;
  cfg.horizon = horizon;
  cfg.include_user = 1;
  cfg.sampler = MPMI_SAMPLER_UNIFORM;
  for (int j = 0; j < MPMI_MAX_NU; ++j) {
    cfg.input_lo[j] = -1.0;
    cfg.input_hi[j] = 1.0;
  }
  cfg.seed = seed;
  if (check(mpmi_session_open(ctx, model, &cfg, &sess), "session_open")) {
    status = 2;
    goto done;
  }
  for (int32_t t = 0; t < n_ticks; ++t) {
    double x_t[4], u_h;
    if (read_exact(f, x_t, sizeof x_t) || read_exact(f, &u_h, sizeof u_h)) {
      fprintf(stderr, "short tick record\n");
      status = 1;
      goto done;
    }
    mpmi_result r;
    if (check(mpmi_evaluate_candidates(sess, x_t, &u_h, NULL, (uint64_t)t, NULL),
              "evaluate_candidates") ||
        check(mpmi_select_input(sess, &r), "select_input")) {
      status = 2;
      goto done;
    }
    uint32_t cost_bits;
    memcpy(&cost_bits, &r.cost, sizeof cost_bits);
    printf("tick %d %d %d %d %d %.17g %" PRIu32 " %" PRIu64 "\n", t, r.index, r.status, r.n_safe,
           r.ttv, r.u_r[0], cost_bits, r.executed_steps);
  }
done:
  if (sess) mpmi_session_close(sess);
  if (model) mpmi_model_free(model);
  if (ctx) mpmi_destroy(ctx);
  fclose(f);
  free(x);
  free(u);
  free(xn);
  return status;
}
