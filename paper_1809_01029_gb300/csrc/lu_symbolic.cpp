// Symbolic phase of the Newton-matrix LU (lu.cu), once per mechanism handle:
// the pivot order, the fill pattern of LU without pivoting in that order,
// and the index tables the factor and solve kernels walk.
//
//  * Order: the species block by greedy minimum degree on the symmetrised
//    pattern (repeatedly the remaining species with the fewest remaining
//    neighbours in the elimination graph, ties by lowest index; its
//    remaining neighbours become a clique), then T and S, whose rows and
//    columns are dense.  perm[k] is the state-vector index of pivot k.
//  * Fill: A = P M P^T; eliminating pivot k joins every row i > k of its
//    column to every column j > k of its row.
//  * Storage (per state, value index e): the strictly lower rows k = 0..N-1
//    (columns ascending), then the upper rows k = N-1..0, each as 1/U_kk
//    followed by U_kj, j > k ascending: the order in which forward and
//    backward substitution read them.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "pj_internal.h"

namespace pj {

namespace {

using Bits = std::vector<uint64_t>;

inline bool bit(const Bits& b, int i) { return (b[i >> 6] >> (i & 63)) & 1u; }
inline void set_bit(Bits& b, int i) { b[i >> 6] |= uint64_t(1) << (i & 63); }

int popcount_and(const Bits& a, const Bits& b) {
  int c = 0;
  for (size_t w = 0; w < a.size(); w++) c += __builtin_popcountll(a[w] & b[w]);
  return c;
}

std::vector<int> min_degree_order(int m, std::vector<Bits> adj) {
  const int words = (m + 63) / 64;
  Bits alive(words, 0);
  for (int i = 0; i < m; i++) set_bit(alive, i);
  std::vector<int> order;
  order.reserve(m);
  for (int step = 0; step < m; step++) {
    int best = -1, best_deg = 1 << 30;
    for (int v = 0; v < m; v++) {
      if (!bit(alive, v)) continue;
      const int d = popcount_and(adj[v], alive);
      if (d < best_deg) {
        best_deg = d;
        best = v;
      }
    }
    Bits nb(words);
    for (int w = 0; w < words; w++) nb[w] = adj[best][w] & alive[w];
    for (int a = 0; a < m; a++) {
      if (!bit(nb, a)) continue;
      for (int w = 0; w < words; w++) adj[a][w] |= nb[w];
      adj[a][a >> 6] &= ~(uint64_t(1) << (a & 63));
    }
    alive[best >> 6] &= ~(uint64_t(1) << (best & 63));
    order.push_back(best);
  }
  return order;
}

}  // namespace

int lu_build(pj_mech* m) {
  const int N = m->ns + 1, ns1 = m->ns - 1;
  const int words = (N + 63) / 64;
  // pattern of M (= pattern of J, diagonal included) from the CSR structure
  std::vector<Bits> P(N, Bits(words, 0));
  for (int i = 0; i < N; i++)
    for (int e = m->csr_ptr[i]; e < m->csr_ptr[i + 1]; e++) set_bit(P[i], m->csr_idx[e]);
  // species block, symmetrised, without the diagonal
  const int swords = (ns1 + 63) / 64;
  std::vector<Bits> S(ns1, Bits(swords > 0 ? swords : 1, 0));
  for (int i = 0; i < ns1; i++)
    for (int j = 0; j < ns1; j++)
      if (i != j && (bit(P[i + 2], j + 2) || bit(P[j + 2], i + 2))) set_bit(S[i], j);
  std::vector<int> order = ns1 > 0 ? min_degree_order(ns1, S) : std::vector<int>();
  std::vector<int32_t>& perm = m->lu_perm;
  perm.clear();
  for (int k : order) perm.push_back(2 + k);
  perm.push_back(0);
  perm.push_back(1);
  std::vector<int32_t> pinv(N);
  for (int k = 0; k < N; k++) pinv[perm[k]] = k;

  // F in pivot order, then the fill of elimination
  std::vector<Bits> F(N, Bits(words, 0));
  for (int k = 0; k < N; k++)
    for (int l = 0; l < N; l++)
      if (bit(P[perm[k]], perm[l])) set_bit(F[k], l);
  for (int k = 0; k < N; k++) {
    Bits upper = F[k];  // row k restricted to columns > k
    for (int j = 0; j <= k; j++) upper[j >> 6] &= ~(uint64_t(1) << (j & 63));
    for (int i = k + 1; i < N; i++)
      if (bit(F[i], k))
        for (int w = 0; w < words; w++) F[i][w] |= upper[w];
  }

  // per-pivot column rows and row columns
  std::vector<int32_t> rptr(N + 1, 0), ridx, cptr(N + 1, 0), cidx;
  for (int k = 0; k < N; k++) {
    for (int i = k + 1; i < N; i++)
      if (bit(F[i], k)) ridx.push_back(i);
    for (int j = k + 1; j < N; j++)
      if (bit(F[k], j)) cidx.push_back(j);
    rptr[k + 1] = (int32_t)ridx.size();
    cptr[k + 1] = (int32_t)cidx.size();
  }
  // CSR entry -> dense pivot-order position
  // dense arrays of the factorisation: rows of an odd number of entries, so
  // that the vector accesses of one column spread over the shared-memory banks
  const int NP = N | 1;
  std::vector<int32_t> m2d(m->nnz);
  for (int i = 0; i < N; i++)
    for (int e = m->csr_ptr[i]; e < m->csr_ptr[i + 1]; e++) m2d[e] = pinv[i] * NP + pinv[m->csr_idx[e]];
  // storage order
  m->lu_rows.clear();
  m->lu_cols.clear();
  std::vector<int32_t> lptr(N + 1, 0), uptr(N + 1, 0);
  for (int k = 0; k < N; k++) {
    for (int j = 0; j < k; j++)
      if (bit(F[k], j)) {
        m->lu_rows.push_back(k);
        m->lu_cols.push_back(j);
      }
    lptr[k + 1] = (int32_t)m->lu_rows.size();
  }
  const int nl = (int)m->lu_rows.size();
  for (int q = 0; q < N; q++) {
    const int k = N - 1 - q;
    uptr[q] = (int32_t)m->lu_rows.size();
    m->lu_rows.push_back(k);
    m->lu_cols.push_back(k);
    for (int j = k + 1; j < N; j++)
      if (bit(F[k], j)) {
        m->lu_rows.push_back(k);
        m->lu_cols.push_back(j);
      }
  }
  uptr[N] = (int32_t)m->lu_rows.size();
  const int lu_nnz = (int)m->lu_rows.size();
  std::vector<int32_t> l2d(lu_nnz), xcol(lu_nnz);
  for (int e = 0; e < lu_nnz; e++) {
    l2d[e] = m->lu_rows[e] * NP + m->lu_cols[e];
    xcol[e] = perm[m->lu_cols[e]];
  }

  DevLu& L = m->lu;
  L = DevLu{};
  L.N = N;
  L.NP = NP;
  L.nnz = m->nnz;
  L.lu_nnz = lu_nnz;
  L.nl = nl;
  if (m->device < 0) return PJ_OK;

  // one device allocation for the tables
  const std::vector<int32_t>* parts[] = {&perm, &rptr, &ridx, &cptr, &cidx, &m2d, &l2d, &xcol, &lptr, &uptr};
  size_t off[10], total = 0;
  for (int p = 0; p < 10; p++) {
    off[p] = total;
    total += (parts[p]->size() * sizeof(int32_t) + 255) & ~size_t(255);
  }
  std::vector<char> blob(total > 0 ? total : 256, 0);
  for (int p = 0; p < 10; p++)
    if (!parts[p]->empty()) std::memcpy(blob.data() + off[p], parts[p]->data(), parts[p]->size() * sizeof(int32_t));
  void* d = nullptr;
  int rc;
  if ((rc = check_cuda(cudaMalloc(&d, blob.size()), "cudaMalloc(LU tables)"))) return rc;
  if ((rc = check_cuda(cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice), "cudaMemcpy(LU tables)"))) {
    cudaFree(d);
    return rc;
  }
  m->lu_blob = d;
  const char* b = static_cast<const char*>(d);
  auto at = [&](int p) { return reinterpret_cast<const int32_t*>(b + off[p]); };
  L.perm = at(0);
  L.rptr = at(1);
  L.ridx = at(2);
  L.cptr = at(3);
  L.cidx = at(4);
  L.m2d = at(5);
  L.l2d = at(6);
  L.xcol = at(7);
  L.lptr = at(8);
  L.uptr = at(9);
  L.dbg = m->dm.dbg;
  return PJ_OK;
}

}  // namespace pj
