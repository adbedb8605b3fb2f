// Standalone driver of the library's host factorisation (factor.cpp) for the CPU tests.
//
//   factor_harness <in> <out>
// in : int32 n, int64 nnz, int64 ptr[n+1], int32 col[nnz], double val[nnz], double xyz[3n]
//      (a symmetric CSR matrix with both triangles, and the vertex coordinates)
// out: int32 n, int64 nnz_L, int32 perm[n], int32 parent[n],
//      int64 S.ptr[n+1], int32 S.col[nnz_S], double S.val[nnz_S]   (S = L^{-1} by rows)
//      int64 St.ptr[n+1], int32 St.col[nnz_S], double St.val[nnz_S] (S^T by rows)
// Exit code 3 with the message on stdout if the factorisation rejects the matrix.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../paper_2603_16478_gb300/csrc/internal.h"

namespace {
template <class T>
bool get(FILE* f, T* p, size_t n) {
  return std::fread(p, sizeof(T), n, f) == n;
}
template <class T>
void put(FILE* f, const T* p, size_t n) {
  std::fwrite(p, sizeof(T), n, f);
}
void put_csr(FILE* f, const ncpadj::CsrD& m) {
  put(f, m.ptr.data(), m.ptr.size());
  put(f, m.col.data(), m.col.size());
  put(f, m.val.data(), m.val.size());
}
}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t n = 0;
  int64_t nnz = 0;
  ncpadj::CsrD A;
  std::vector<double> xyz;
  bool ok = get(f, &n, 1) && get(f, &nnz, 1);
  if (ok) {
    A.n = n;
    A.ptr.resize(n + 1);
    A.col.resize(nnz);
    A.val.resize(nnz);
    xyz.resize(3 * (size_t)n);
    ok = get(f, A.ptr.data(), n + 1) && get(f, A.col.data(), nnz) && get(f, A.val.data(), nnz) &&
         get(f, xyz.data(), 3 * (size_t)n);
  }
  std::fclose(f);
  if (!ok) return 2;
  ncpadj::ElasticFactor F;
  try {
    ncpadj::factor_elastic(A, xyz.data(), F);
  } catch (const ncpadj::Error& e) {
    std::printf("%s\n", e.msg.c_str());
    return 3;
  }
  FILE* o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  put(o, &F.n, 1);
  put(o, &F.nnz_L, 1);
  put(o, F.perm.data(), F.perm.size());
  put(o, F.parent.data(), F.parent.size());
  put_csr(o, F.S);
  put_csr(o, F.St);
  std::fclose(o);
  return 0;
}
