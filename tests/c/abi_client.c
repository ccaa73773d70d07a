/*
 * A plain C client of the library's C-ABI (include/qtt.h): it links
 * libqtt.so and, for the expected values, the C oracle (test
 * infrastructure).  Usage:
 *   abi_client host    -- argument validation and host-only calls (no GPU)
 *   abi_client device  -- also: create an operator from seeded cores, apply
 *                         it in FP64 through qtt_apply and compare with the
 *                         oracle's sweep (relative L2 <= 1e-12), and write /
 *                         read it back through the .qtt file.
 * Exit status 0 on success; a message on stderr otherwise.
 */
#include <cuda_runtime_api.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "qtt.h"

/* the oracle's sweep (oracle/qtt_oracle.c) */
int qo_apply(int d, const int *r, const double *G, int64_t nrhs, const double *x, int64_t ldx,
             double *y, int64_t ldy, int threads);

#define CHECK(cond, ...)                    \
  do {                                      \
    if (!(cond)) {                          \
      fprintf(stderr, "abi_client: ");      \
      fprintf(stderr, __VA_ARGS__);         \
      fprintf(stderr, "\n");                \
      return 1;                             \
    }                                       \
  } while (0)

/* SplitMix64 to uniform in [-1, 1) */
static uint64_t g_state = 0x9E3779B97F4A7C15ull;
static double next_uniform(void) {
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static int host_checks(void) {
  qtt_op *A = NULL;
  const int bad_ranks[3] = {2, 3, 1};
  const double cores[64] = {0};
  const double *core_ptrs[2] = {cores, NULL};
  CHECK(qtt_create_flat(&A, 2, bad_ranks, cores, 0, NULL) == QTT_ERR_INVALID_ARG,
        "qtt_create_flat accepted ranks[0] = 2");
  CHECK(A == NULL, "qtt_create_flat left a handle after failing");
  CHECK(qtt_create(&A, 0, bad_ranks, core_ptrs, 0, NULL) == QTT_ERR_INVALID_ARG,
        "d = 0 accepted");
  {
    const int ranks[3] = {1, 2, 1};
    CHECK(qtt_create(&A, 2, ranks, core_ptrs, 0, NULL) == QTT_ERR_INVALID_ARG,
          "qtt_create accepted a NULL core pointer");
  }
  CHECK(qtt_destroy(NULL) == QTT_OK, "qtt_destroy(NULL) failed");
  CHECK(strcmp(qtt_status_string(QTT_OK), "ok") == 0, "status string of QTT_OK");
  CHECK(qtt_apply(NULL, NULL, NULL, 1, 1, QTT_F64, QTT_F64, NULL) == QTT_ERR_INVALID_ARG,
        "qtt_apply accepted a NULL operator");
  CHECK(qtt_apply_host(NULL, NULL, NULL, 1, 1, QTT_F64, QTT_F64, 0, NULL) ==
            QTT_ERR_INVALID_ARG,
        "qtt_apply_host accepted a NULL operator");
  CHECK(qtt_batch_run_host(NULL, NULL, NULL, NULL) == QTT_ERR_INVALID_ARG,
        "qtt_batch_run_host accepted a NULL batch");
  CHECK(strlen(qtt_last_error()) > 0, "no message after a failing call");
  return 0;
}

static int device_checks(const char *tmpdir) {
  enum { D = 11, NRHS = 3 };
  int ranks[D + 1];
  for (int k = 0; k <= D; ++k) {
    int r = 1 << (k < D - k ? k : D - k);
    ranks[k] = r < 12 ? r : 12;
  }
  int64_t np = 0;
  for (int k = 0; k < D; ++k) np += 4 * (int64_t)ranks[k] * ranks[k + 1];
  const int64_t N = (int64_t)1 << D;
  double *cores = malloc(sizeof(double) * np);
  double *x = malloc(sizeof(double) * N * NRHS), *y = malloc(sizeof(double) * N * NRHS);
  double *ref = malloc(sizeof(double) * N * NRHS);
  CHECK(cores && x && y && ref, "host allocation");
  for (int64_t e = 0; e < np; ++e) cores[e] = next_uniform() * 0.3;
  for (int64_t e = 0; e < N * NRHS; ++e) x[e] = next_uniform();

  /* the per-core form of qtt_create: one pointer per core */
  const double *core_ptrs[D];
  {
    int64_t off = 0;
    for (int k = 0; k < D; ++k) {
      core_ptrs[k] = cores + off;
      off += 4 * (int64_t)ranks[k] * ranks[k + 1];
    }
  }
  qtt_op *A = NULL;
  CHECK(qtt_create(&A, D, ranks, core_ptrs, 0, NULL) == QTT_OK, "qtt_create: %s",
        qtt_last_error());
  CHECK(qtt_op_d(A) == D && qtt_op_rank(A, 5) == ranks[5], "operator queries");
  double *xd = NULL, *yd = NULL;
  CHECK(cudaMalloc((void **)&xd, sizeof(double) * N * NRHS) == cudaSuccess, "cudaMalloc x");
  CHECK(cudaMalloc((void **)&yd, sizeof(double) * N * NRHS) == cudaSuccess, "cudaMalloc y");
  CHECK(cudaMemcpy(xd, x, sizeof(double) * N * NRHS, cudaMemcpyHostToDevice) == cudaSuccess,
        "upload x");
  CHECK(qtt_apply(A, xd, yd, NRHS, N, QTT_F64, QTT_F64, NULL) == QTT_OK, "qtt_apply: %s",
        qtt_last_error());
  CHECK(qtt_sync_status(NULL) == QTT_OK, "qtt_sync_status: %s", qtt_last_error());
  CHECK(cudaMemcpy(y, yd, sizeof(double) * N * NRHS, cudaMemcpyDeviceToHost) == cudaSuccess,
        "download y");
  CHECK(qo_apply(D, ranks, cores, NRHS, x, N, ref, N, 1) == 0, "oracle apply");
  double num = 0.0, den = 0.0;
  for (int64_t e = 0; e < N * NRHS; ++e) {
    num += (y[e] - ref[e]) * (y[e] - ref[e]);
    den += ref[e] * ref[e];
  }
  CHECK(den > 0.0 && sqrt(num / den) <= 1e-12, "FP64 apply vs oracle: rel L2 %.3e",
        sqrt(num / den));

  /* the .qtt file round trip gives the same cores */
  char path[4096];
  snprintf(path, sizeof(path), "%s/abi_client.qtt", tmpdir);
  CHECK(qtt_write_file(path, D, ranks, cores) == QTT_OK, "qtt_write_file: %s", qtt_last_error());
  int d2 = 0, r2[D + 1];
  int64_t n2 = 0;
  CHECK(qtt_read_file(path, &d2, NULL, 0, NULL, 0, &n2) == QTT_OK && d2 == D && n2 == np,
        "qtt_read_file sizes");
  double *c2 = malloc(sizeof(double) * np);
  CHECK(c2 && qtt_read_file(path, &d2, r2, D + 1, c2, np, &n2) == QTT_OK, "qtt_read_file");
  CHECK(memcmp(c2, cores, sizeof(double) * np) == 0 && memcmp(r2, ranks, sizeof(ranks)) == 0,
        "file round trip changed the operator");
  CHECK(qtt_destroy(A) == QTT_OK, "qtt_destroy");
  cudaFree(xd);
  cudaFree(yd);
  free(cores); free(x); free(y); free(ref); free(c2);
  printf("abi_client device ok: d=%d nrhs=%d rel L2 %.2e\n", D, NRHS, sqrt(num / den));
  return 0;
}

int main(int argc, char **argv) {
  const int device = argc > 1 && strcmp(argv[1], "device") == 0;
  if (host_checks() != 0) return 1;
  printf("abi_client host ok\n");
  if (device) return device_checks(argc > 2 ? argv[2] : ".");
  return 0;
}
