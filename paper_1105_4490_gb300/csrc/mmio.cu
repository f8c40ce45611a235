// Matrix Market input and output (host): the exchange format of the sparse
// matrix collections the paper orders.  Coordinate files of any field (real,
// integer, complex as its modulus, pattern as 1) and symmetry (general,
// symmetric, skew-symmetric, hermitian) are read into a row-major CSR with
// sorted columns and duplicate entries summed; symmetric storage can be
// expanded to both triangles.  Host code only: the result is the input of
// vmo_build_hypergraph after a copy to the device.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "vmo_internal.cuh"

namespace vmo {
namespace {

struct Entry {
  int32_t r, c;
  float v;
};

std::string lower(const char* s) {
  std::string o(s);
  for (char& ch : o) ch = (char)std::tolower((unsigned char)ch);
  return o;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

}  // namespace
}  // namespace vmo

using namespace vmo;

extern "C" void vmo_free_host_csr(vmo_host_csr* csr) {
  if (!csr) return;
  free(csr->rowptr);
  free(csr->colidx);
  free(csr->values);
  csr->rowptr = nullptr;
  csr->colidx = nullptr;
  csr->values = nullptr;
  csr->m = csr->n = 0;
  csr->nnz = 0;
}

extern "C" vmo_status vmo_read_matrix_market(const char* path, int32_t expand_symmetric, vmo_host_csr* out) {
  if (!path || !out) return invalid("null argument");
  memset(out, 0, sizeof(*out));
  File file;
  file.f = fopen(path, "r");
  if (!file.f) return invalid(std::string("cannot open ") + path);
  char line[4096];
  if (!fgets(line, sizeof(line), file.f)) return invalid("empty file");
  char banner[64] = {0}, object[64] = {0}, format[64] = {0}, field[64] = {0}, symmetry[64] = {0};
  if (sscanf(line, "%63s %63s %63s %63s %63s", banner, object, format, field, symmetry) != 5 ||
      lower(banner) != "%%matrixmarket")
    return invalid("not a Matrix Market file (banner)");
  if (lower(object) != "matrix" || lower(format) != "coordinate")
    return unsupported("only coordinate matrices are read");
  const std::string fld = lower(field), sym = lower(symmetry);
  const bool pattern = fld == "pattern", complex_ = fld == "complex";
  if (!pattern && !complex_ && fld != "real" && fld != "integer" && fld != "double")
    return invalid("unknown field " + fld);
  const bool general = sym == "general", skew = sym == "skew-symmetric";
  if (!general && !skew && sym != "symmetric" && sym != "hermitian") return invalid("unknown symmetry " + sym);
  long long m = -1, n = -1, nz = -1;
  while (fgets(line, sizeof(line), file.f)) {
    if (line[0] == '%') continue;
    char* p = line;
    while (*p && std::isspace((unsigned char)*p)) ++p;
    if (!*p) continue;
    if (sscanf(p, "%lld %lld %lld", &m, &n, &nz) != 3) return invalid("bad size line");
    break;
  }
  if (m < 0 || n < 0 || nz < 0) return invalid("missing size line");
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || nz > (long long)INT32_MAX / 2) return unsupported("matrix too large");
  if (!general && m != n) return invalid("symmetric storage needs a square matrix");
  std::vector<Entry> e;
  e.reserve((size_t)(general || !expand_symmetric ? nz : 2 * nz));
  for (long long k = 0; k < nz; ++k) {
    if (!fgets(line, sizeof(line), file.f)) return invalid("file ends before all entries are read");
    if (line[0] == '%') {
      --k;
      continue;
    }
    char* p = line;
    char* q = nullptr;
    const long long i = strtoll(p, &q, 10);
    if (q == p) return invalid("bad entry line");
    p = q;
    const long long j = strtoll(p, &q, 10);
    if (q == p) return invalid("bad entry line");
    p = q;
    double v = 1.0;
    if (!pattern) {
      v = strtod(p, &q);
      if (q == p) return invalid("bad entry value");
      if (complex_) {  // the modulus stands for a complex entry
        p = q;
        const double im = strtod(p, &q);
        if (q == p) return invalid("bad entry value");
        v = std::sqrt(v * v + im * im);
      }
    }
    if (i < 1 || i > m || j < 1 || j > n) return invalid("entry index outside the matrix");
    const int32_t r = (int32_t)(i - 1), c = (int32_t)(j - 1);
    e.push_back({r, c, (float)v});
    if (!general && expand_symmetric && r != c) e.push_back({c, r, (float)(skew ? -v : v)});
  }
  std::sort(e.begin(), e.end(), [](const Entry& a, const Entry& b) { return a.r != b.r ? a.r < b.r : a.c < b.c; });
  // duplicates summed
  size_t u = 0;
  for (size_t k = 0; k < e.size(); ++k) {
    if (u > 0 && e[u - 1].r == e[k].r && e[u - 1].c == e[k].c) {
      e[u - 1].v += e[k].v;
    } else {
      e[u++] = e[k];
    }
  }
  e.resize(u);
  out->m = (int32_t)m;
  out->n = (int32_t)n;
  out->nnz = (int64_t)u;
  out->rowptr = (int32_t*)calloc((size_t)m + 1, sizeof(int32_t));
  out->colidx = (int32_t*)malloc(std::max<size_t>(u, 1) * sizeof(int32_t));
  out->values = (float*)malloc(std::max<size_t>(u, 1) * sizeof(float));
  if (!out->rowptr || !out->colidx || !out->values) {
    vmo_free_host_csr(out);
    return VMO_ERR_OOM;
  }
  for (size_t k = 0; k < u; ++k) {
    out->rowptr[e[k].r + 1]++;
    out->colidx[k] = e[k].c;
    out->values[k] = e[k].v;
  }
  for (long long i = 0; i < m; ++i) out->rowptr[i + 1] += out->rowptr[i];
  return VMO_OK;
}

extern "C" vmo_status vmo_write_matrix_market(const char* path, const vmo_host_csr* csr, int32_t pattern) {
  if (!path || !csr || csr->m < 0 || csr->n < 0 || !csr->rowptr) return invalid("null or negative argument");
  if (csr->nnz > 0 && (!csr->colidx || (!pattern && !csr->values))) return invalid("null entry arrays");
  File file;
  file.f = fopen(path, "w");
  if (!file.f) return invalid(std::string("cannot create ") + path);
  fprintf(file.f, "%%%%MatrixMarket matrix coordinate %s general\n", pattern ? "pattern" : "real");
  fprintf(file.f, "%d %d %lld\n", csr->m, csr->n, (long long)csr->nnz);
  for (int32_t i = 0; i < csr->m; ++i)
    for (int32_t t = csr->rowptr[i]; t < csr->rowptr[i + 1]; ++t) {
      if (pattern)
        fprintf(file.f, "%d %d\n", i + 1, csr->colidx[t] + 1);
      else
        fprintf(file.f, "%d %d %.9g\n", i + 1, csr->colidx[t] + 1, (double)csr->values[t]);
    }
  if (ferror(file.f)) return invalid(std::string("write failed: ") + path);
  return VMO_OK;
}
