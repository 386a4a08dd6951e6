// Host construction of the plane-wave layout and FFT plans.
//
// Gamma-point storage (paper Sec. 2.1 works with real orbitals at Gamma): the caller gives the
// half sphere; internally every G is assigned to a "rep column" (n1, n2) with n1 > 0, or
// n1 = 0 and n2 > 0, or the column (0, 0). A half-sphere G whose own column is not a rep column
// is stored as conj(f(G)) at -G, which lies in a rep column. Column (0, 0) is stored in full
// (f(0,0,-z) = conj f(0,0,z)). Each rep column holds the contiguous n3 interval of the sphere in
// that column, so one vector is the concatenation of those intervals.
#include <cmath>
#include <map>
#include <set>
#include <utility>

#include "engine.cuh"

namespace wdf {

// Device memory held by the library's grow-only buffers (all contexts and models of the
// process), the cudaMalloc calls made for them, and an optional cap on the bytes held
// (wdf_set_device_limit; 0: none). A growth the cap refuses leaves the buffer as it was.
std::atomic<long long> g_dev_bytes{0};
std::atomic<long long> g_dev_allocs{0};
std::atomic<long long> g_dev_cap{0};

void DBuf::ensure(size_t bytes) {
  if (bytes <= cap) return;
  const long long limit = g_dev_cap.load();
  if (limit > 0 && g_dev_bytes.load() - (long long)cap + (long long)bytes > limit)
    throw ApiFailure(WDF_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes refused: the library holds " +
                                     std::to_string(g_dev_bytes.load()) + " of its limit of " + std::to_string(limit) + " bytes");
  if (p) {
    cudaError_t e = cudaFree(p);
    p = nullptr;
    g_dev_bytes.fetch_sub((long long)cap);
    cap = 0;
    if (e != cudaSuccess) throw CudaFailure(e, "cudaFree", __FILE__, __LINE__);
  }
  if (bytes == 0) return;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    p = nullptr;
    (void)cudaGetLastError();
    throw ApiFailure(WDF_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  g_dev_allocs.fetch_add(1);
  g_dev_bytes.fetch_add((long long)bytes);
  cap = bytes;
}

void DBuf::release() {
  if (p) {
    (void)cudaFree(p);
    g_dev_bytes.fetch_sub((long long)cap);
  }
  p = nullptr;
  cap = 0;
}

Plan1D make_plan(int n) {
  Plan1D P{};
  P.n = n;
  int m = n, k = 0;
  const int radices[4] = {4, 2, 3, 5};
  for (int ri = 0; ri < 4; ++ri) {
    while (m % radices[ri] == 0) {
      if (k >= kMaxStages) throw ApiFailure(WDF_EINVAL, "FFT length has too many factors");
      P.r[k++] = radices[ri];
      m /= radices[ri];
    }
  }
  if (m != 1) throw ApiFailure(WDF_EINVAL, "FFT length " + std::to_string(n) + " is not a product of 2, 3 and 5");
  P.nst = k;
  P.L[0] = 1;
  for (int j = 0; j < k; ++j) P.L[j + 1] = P.L[j] * P.r[j];
  return P;
}

// pos(v) = (v mod r_k) n / r_k + pos'(v div r_k), pos' the map of the first k-1 radices
std::vector<int> digit_reversal(const Plan1D &P) {
  std::vector<int> pos(P.n);
  for (int v = 0; v < P.n; ++v) {
    int val = v, N = P.n, acc = 0;
    for (int j = P.nst - 1; j >= 0; --j) {
      const int r = P.r[j];
      const int M = N / r;
      acc += (val % r) * M;
      val /= r;
      N = M;
    }
    pos[v] = acc;
  }
  return pos;
}

static int wrapi(int z, int n) {
  int m = z % n;
  return m < 0 ? m + n : m;
}

Layout build_layout(const int32_t *miller, int npw_h, const int n[3], const double bvec[9]) {
  Layout L;
  if (npw_h < 1) throw ApiFailure(WDF_EINVAL, "npw_h must be positive");
  for (int a = 0; a < 3; ++a)
    if (n[a] < 2 || n[a] > kMaxN) throw ApiFailure(WDF_EINVAL, "grid sizes must lie in [2, 128]");
  L.P1 = make_plan(n[0]);
  L.P2 = make_plan(n[1]);
  L.P3 = make_plan(n[2]);
  if (miller[0] != 0 || miller[1] != 0 || miller[2] != 0) throw ApiFailure(WDF_EINVAL, "the first Miller triple must be G = 0");

  // half-sphere check and assignment to rep columns
  std::set<std::tuple<int, int, int>> seen;
  std::map<std::pair<int, int>, std::vector<int>> colz;  // rep column -> n3 values
  struct Assign {
    int c1, c2, z;
    bool conj;
  };
  std::vector<Assign> asg(npw_h);
  for (int i = 0; i < npw_h; ++i) {
    const int a = miller[3 * i], b = miller[3 * i + 1], z = miller[3 * i + 2];
    if (2 * std::abs(a) + 1 > n[0] || 2 * std::abs(b) + 1 > n[1] || 2 * std::abs(z) + 1 > n[2])
      throw ApiFailure(WDF_EINVAL, "grid too small for the plane-wave sphere (need n >= 2 |m| + 1 on every axis)");
    if (!seen.insert({a, b, z}).second) throw ApiFailure(WDF_EINVAL, "duplicate Miller triple");
    if (i > 0 && seen.count({-a, -b, -z})) throw ApiFailure(WDF_EINVAL, "Miller set holds both G and -G");
    Assign s;
    if (a > 0 || (a == 0 && b > 0)) s = {a, b, z, false};
    else if (a < 0 || (a == 0 && b < 0)) s = {-a, -b, -z, true};
    else s = {0, 0, z, false};
    asg[i] = s;
    auto &v = colz[{s.c1, s.c2}];
    v.push_back(s.z);
    if (s.c1 == 0 && s.c2 == 0 && z != 0) v.push_back(-z);
  }
  if (!colz.count({0, 0})) throw ApiFailure(WDF_EINVAL, "missing column (0, 0)");
  // columns: (0,0) first, then sorted by (n1, n2)
  std::vector<std::pair<int, int>> cols;
  cols.push_back({0, 0});
  for (auto &kv : colz)
    if (!(kv.first.first == 0 && kv.first.second == 0)) cols.push_back(kv.first);
  L.K = (int)cols.size();
  std::map<std::pair<int, int>, int> colidx;
  L.col_off.assign(L.K + 1, 0);
  for (int k = 0; k < L.K; ++k) {
    auto &zs = colz[cols[k]];
    std::sort(zs.begin(), zs.end());
    for (size_t t = 1; t < zs.size(); ++t)
      if (zs[t] != zs[t - 1] + 1) throw ApiFailure(WDF_EINVAL, "n3 values of a column do not form one interval");
    colidx[cols[k]] = k;
    L.col_n1.push_back(cols[k].first);
    L.col_n2.push_back(cols[k].second);
    L.col_zlo.push_back(zs.front());
    L.col_off[k + 1] = L.col_off[k] + (int)zs.size();
  }
  L.nint = L.col_off[L.K];
  L.len0 = L.col_off[1];
  L.ld = ((L.nint + 31) / 32) * 32;
  L.ndisk = 2 * L.K - 1;
  L.ldcb = ((L.ndisk + 7) / 8) * 8;
  L.e_col.resize(L.nint);
  L.e_z.resize(L.nint);
  L.g2.assign(L.ld, 0.0);
  L.vhalf.assign(L.ld, 0.0);
  for (int k = 0; k < L.K; ++k) {
    for (int e = L.col_off[k]; e < L.col_off[k + 1]; ++e) {
      const int z = L.col_zlo[k] + (e - L.col_off[k]);
      L.e_col[e] = k;
      L.e_z[e] = z;
      double gx = 0, gy = 0, gz = 0;
      const int m3[3] = {L.col_n1[k], L.col_n2[k], z};
      for (int a = 0; a < 3; ++a) {
        gx += m3[a] * bvec[3 * a + 0];
        gy += m3[a] * bvec[3 * a + 1];
        gz += m3[a] * bvec[3 * a + 2];
      }
      const double g2 = gx * gx + gy * gy + gz * gz;
      L.g2[e] = g2;
      L.vhalf[e] = (k == 0 && z == 0) ? 0.0 : std::sqrt(4.0 * M_PI / g2);
    }
  }
  // external maps
  L.emap.resize(npw_h);
  L.emap2.assign(npw_h, -1);
  L.econj.resize(npw_h);
  for (int i = 0; i < npw_h; ++i) {
    const Assign &s = asg[i];
    const int k = colidx[{s.c1, s.c2}];
    L.emap[i] = L.col_off[k] + (s.z - L.col_zlo[k]);
    L.econj[i] = s.conj ? 1 : 0;
    if (k == 0 && s.z != 0) L.emap2[i] = L.col_off[0] + (-s.z - L.col_zlo[0]);
  }
  // disk columns and plane tile positions
  const std::vector<int> pos1 = digit_reversal(L.P1), pos2 = digit_reversal(L.P2), pos3 = digit_reversal(L.P3);
  const int pitch = n[0] + 1;
  L.tile_idx.resize(L.ndisk);
  L.jidx.assign((size_t)n[0] * n[1], -1);
  L.jnat.assign(L.ndisk, 0);
  std::set<int> xs, xsn;
  for (int j = 0; j < L.ndisk; ++j) {
    int a, b;
    if (j < L.K) {
      a = L.col_n1[j];
      b = L.col_n2[j];
    } else {
      a = -L.col_n1[j - L.K + 1];
      b = -L.col_n2[j - L.K + 1];
    }
    const int x = pos1[wrapi(a, n[0])], y = pos2[wrapi(b, n[1])];
    L.tile_idx[j] = y * pitch + x;
    xs.insert(x);
    xsn.insert(wrapi(a, n[0]));
    L.jidx[(size_t)wrapi(b, n[1]) * n[0] + wrapi(a, n[0])] = j;
    L.jnat[j] = wrapi(b, n[1]) * n[0] + wrapi(a, n[0]);
    L.xmax = std::max(L.xmax, std::abs(a));
    L.ymax = std::max(L.ymax, std::abs(b));
  }
  L.xact.assign(xs.begin(), xs.end());
  L.xactn.assign(xsn.begin(), xsn.end());
  L.pos3.resize(n[2]);
  for (int t = 0; t < n[2]; ++t) L.pos3[t] = (short)pos3[t];
  return L;
}

}  // namespace wdf
