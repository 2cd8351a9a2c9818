// Model files: the parameters of a handle (r_in, r_cut, the snapshot lists,
// K2/K3/K4, P3/P4), its projection Q and optionally the coefficients c of a
// fitted linear model, as versioned text with every number in round-trip
// precision.  The paper ships no model format; a model saved here and loaded
// again evaluates bit for bit like the handle it came from (same parameters,
// same Q, same c).
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pod_internal.h"

using namespace fastpod;

namespace {
constexpr const char* MAGIC = "fastpod-model";
constexpr int VERSION = 1;

void put_list(FILE* f, const char* key, const std::vector<double>& v) {
  std::fprintf(f, "%s %zu", key, v.size());
  for (double x : v) std::fprintf(f, " %.17g", x);
  std::fprintf(f, "\n");
}

// Reads "key n v1 .. vn" (n <= nmax); false on a mismatch.
bool get_list(FILE* f, const char* key, std::vector<double>& v, size_t nmax) {
  char word[64];
  size_t n = 0;
  if (std::fscanf(f, "%63s %zu", word, &n) != 2 || std::strcmp(word, key) != 0 || n > nmax) return false;
  v.resize(n);
  for (size_t k = 0; k < n; ++k) {
    char num[64];
    if (std::fscanf(f, "%63s", num) != 1) return false;
    char* end = nullptr;
    errno = 0;
    v[k] = std::strtod(num, &end);
    if (errno != 0 || !end || *end != '\0' || !std::isfinite(v[k])) return false;
  }
  return true;
}

bool get_ints(FILE* f, const char* key, int* out, int n) {
  char word[64];
  if (std::fscanf(f, "%63s", word) != 1 || std::strcmp(word, key) != 0) return false;
  for (int k = 0; k < n; ++k)
    if (std::fscanf(f, "%d", &out[k]) != 1) return false;
  return true;
}
}  // namespace

extern "C" int pod_save(const pod_handle* h, const char* path, const double* c) {
  if (!h || !path) return POD_EINVAL;
  pod_handle* hm = const_cast<pod_handle*>(h);
  if (c)
    for (int m = 0; m < h->M; ++m)
      if (!std::isfinite(c[m])) return hm->fail(POD_EINVAL, "coefficients must be finite");
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return hm->fail(POD_EIO, "cannot write %s", tmp.c_str());
  const HostParams& P = h->P;
  std::fprintf(f, "%s %d\n", MAGIC, VERSION);
  std::fprintf(f, "r_in %.17g\nr_cut %.17g\n", P.r_in, P.r_cut);
  put_list(f, "alpha", P.alpha);
  put_list(f, "beta", P.beta);
  put_list(f, "gamma", P.gamma);
  std::fprintf(f, "modes %d %d %d\ndegrees %d %d\n", P.K2, P.K3, P.K4, P.P3, P.P4);
  std::fprintf(f, "shape %d %d\n", h->Ns, h->K);
  put_list(f, "Q", h->Q);
  if (c)
    put_list(f, "c", std::vector<double>(c, c + h->M));
  else
    std::fprintf(f, "c 0\n");
  std::fprintf(f, "end\n");
  const bool ok = std::fflush(f) == 0 && !std::ferror(f);
  if (std::fclose(f) != 0 || !ok) {
    std::remove(tmp.c_str());
    return hm->fail(POD_EIO, "cannot write %s", tmp.c_str());
  }
  if (std::rename(tmp.c_str(), path) != 0) {  // the file appears whole or not at all
    std::remove(tmp.c_str());
    return hm->fail(POD_EIO, "cannot write %s", path);
  }
  return POD_OK;
}

extern "C" int pod_load(const char* path, int precision, pod_handle** out, double* c_out, int c_capacity,
                        int* n_c) {
  if (!path || !out) return POD_EINVAL;
  *out = nullptr;
  if (n_c) *n_c = 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return POD_EIO;
  char word[64];
  int version = 0;
  bool ok = std::fscanf(f, "%63s %d", word, &version) == 2 && std::strcmp(word, MAGIC) == 0 && version == VERSION;
  double r_in = 0, r_cut = 0;
  ok = ok && std::fscanf(f, "%63s %lf", word, &r_in) == 2 && std::strcmp(word, "r_in") == 0;
  ok = ok && std::fscanf(f, "%63s %lf", word, &r_cut) == 2 && std::strcmp(word, "r_cut") == 0;
  std::vector<double> alpha, beta, gamma, Q, c;
  int modes[3] = {0, 0, 0}, degrees[2] = {-1, -1}, shape[2] = {0, 0};
  ok = ok && get_list(f, "alpha", alpha, 64) && get_list(f, "beta", beta, 64) && get_list(f, "gamma", gamma, 64);
  ok = ok && get_ints(f, "modes", modes, 3) && get_ints(f, "degrees", degrees, 2) && get_ints(f, "shape", shape, 2);
  ok = ok && shape[0] > 0 && shape[1] > 0 && shape[0] <= 64 && shape[1] <= 64;
  ok = ok && get_list(f, "Q", Q, 4096) && Q.size() == (size_t)shape[0] * shape[1];
  ok = ok && get_list(f, "c", c, 4096);
  ok = ok && std::fscanf(f, "%63s", word) == 1 && std::strcmp(word, "end") == 0;
  std::fclose(f);
  if (!ok) return POD_EINVAL;
  pod_params prm{};
  prm.r_in = r_in;
  prm.r_cut = r_cut;
  prm.n_alpha = (int)alpha.size();
  prm.alpha = alpha.data();
  prm.n_beta = (int)beta.size();
  prm.beta = beta.data();
  prm.n_gamma = (int)gamma.size();
  prm.gamma = gamma.empty() ? nullptr : gamma.data();
  prm.K2 = modes[0];
  prm.K3 = modes[1];
  prm.K4 = modes[2];
  prm.P3 = degrees[0];
  prm.P4 = degrees[1];
  prm.precision = precision;
  prm.Q = Q.data();
  int rc = pod_create(&prm, out);
  if (rc) return rc;  // *out holds the handle with the message (or NULL)
  pod_handle* h = *out;
  if (h->Ns != shape[0] || h->K != shape[1]) return h->fail(POD_EINVAL, "model file: Q has the wrong shape");
  if (!c.empty()) {
    if ((int)c.size() != h->M) return h->fail(POD_EINVAL, "model file: %zu coefficients for M = %d", c.size(), h->M);
    if (c_out && c_capacity < h->M) return h->fail(POD_EINVAL, "c_capacity %d < M = %d", c_capacity, h->M);
    if (c_out) std::memcpy(c_out, c.data(), sizeof(double) * c.size());
    if (n_c) *n_c = h->M;
  }
  return POD_OK;
}
