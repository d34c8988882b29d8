// Problem setup: validation of the inputs, the chaos tables and the sparse G_k
// couplings (Sec. 2, eq. (gPC-u), (global-system); Sec. 3), and the Galerkin
// multigrid hierarchy of the mean-value matrix A_0 used by the inner solves.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>

#include "df64.cuh"
#include "graph.cuh"
#include "sghsc_internal.cuh"

namespace sghsc {

static thread_local char g_err[1024] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

// Graded multi-indices; inside one degree, descending lexicographic order.
static void emit_degree(int M, int pos, int remaining, std::vector<int>& cur, std::vector<int>& out) {
  if (pos == M - 1) {
    cur[pos] = remaining;
    out.insert(out.end(), cur.begin(), cur.end());
    return;
  }
  for (int a = remaining; a >= 0; --a) {
    cur[pos] = a;
    emit_degree(M, pos + 1, remaining - a, cur, out);
  }
}

// E[xi psi_m psi_{m+1}] for the orthonormal 1-D family. Legendre with
// xi ~ U(-sqrt3, sqrt3): sqrt3 (m+1) / sqrt((2m+1)(2m+3)); Hermite with
// xi ~ N(0,1): sqrt(m+1).
static double xi_coupling(int m, int family) {
  if (family == SG_HERMITE) return std::sqrt((double)m + 1.0);
  return std::sqrt(3.0) * (m + 1.0) / std::sqrt((2.0 * m + 1.0) * (2.0 * m + 3.0));
}

template <typename T>
static int upload(T** dst, const T* src, size_t count) {
  if (count == 0) {
    *dst = nullptr;
    return SG_OK;
  }
  SG_TRY_CUDA(cudaMalloc((void**)dst, count * sizeof(T)));
  SG_TRY_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return SG_OK;
}

struct HostEdges {
  std::vector<int> ptr{0}, k, j;
  std::vector<double> c;
};

static int upload_edges(const HostEdges& he, EdgeList& E, int out0 = 0, int in0 = 0, int nin = 0) {
  E.out0 = out0;
  E.in0 = in0;
  E.nin = nin;
  E.nout = (int)he.ptr.size() - 1;
  E.nedges = (int)he.k.size();
  std::vector<float> c32(he.c.begin(), he.c.end());
  // Outputs ordered by their number of couplings, so the lanes of a warp run
  // coupling loops of equal length (equal counts keep column order).
  std::vector<int> perm(E.nout);
  for (int l = 0; l < E.nout; ++l) perm[l] = l;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
    return he.ptr[a + 1] - he.ptr[a] > he.ptr[b + 1] - he.ptr[b];
  });
  SG_TRY(upload(&E.perm, perm.data(), perm.size()));
  SG_TRY(upload(&E.ptr, he.ptr.data(), he.ptr.size()));
  SG_TRY(upload(&E.k, he.k.data(), he.k.size()));
  SG_TRY(upload(&E.j, he.j.data(), he.j.size()));
  SG_TRY(upload(&E.c64, he.c.data(), he.c.size()));
  SG_TRY(upload(&E.c32, c32.data(), c32.size()));
  {
    std::vector<df64> cdf(he.c.size());
    for (size_t t = 0; t < he.c.size(); ++t) cdf[t] = df_split_host(he.c[t]);
    df64* d = nullptr;
    SG_TRY(upload(&d, cdf.data(), cdf.size()));
    E.cdf = d;
  }
  std::map<std::pair<int, int>, int> pairs;
  for (int t = 0; t < E.nedges; ++t) pairs.emplace(std::make_pair(he.k[t], he.j[t]), 0);
  std::vector<int> pk, pj, pair(E.nedges);
  for (auto& kv : pairs) {
    kv.second = (int)pk.size();
    pk.push_back(kv.first.first);
    pj.push_back(kv.first.second);
  }
  for (int t = 0; t < E.nedges; ++t) pair[t] = pairs.at(std::make_pair(he.k[t], he.j[t]));
  E.npair = (int)pk.size();
  {
    // coefficient classes; class 0 is the coefficient 0, which pads the
    // shorter slots of a warp to the warp's longest (a zero word adds 0)
    std::map<double, int> cls;
    for (double c : he.c) cls.emplace(c, 0);
    if (cls.size() + (cls.count(0.0) ? 0 : 1) <= 256 && E.npair < (1 << 24)) {
      std::vector<df64> tab{df64(0.f, 0.f)};
      std::vector<float> tab32{0.f};
      for (auto& kv : cls) {
        if (kv.first == 0.0) continue;
        kv.second = (int)tab.size();
        tab.push_back(df_split_host(kv.first));
        tab32.push_back((float)kv.first);
      }
      SG_TRY(upload(&E.ctab32, tab32.data(), tab32.size()));
      // slot-transposed packing: warp w (slots 32w .. 32w+31, counts sorted
      // descending) takes 32 words per coupling of its first slot
      std::vector<int> tb(E.nout);
      size_t total = 0;
      for (int w0 = 0; w0 < E.nout; w0 += 32) {
        const int cmax = he.ptr[perm[w0] + 1] - he.ptr[perm[w0]];
        for (int sl = w0; sl < std::min(w0 + 32, E.nout); ++sl) tb[sl] = (int)total + (sl - w0);
        total += (size_t)32 * cmax;
      }
      if (total >= (size_t)1 << 31) return SG_ERR_UNSUPPORTED;
      std::vector<unsigned> packed(std::max<size_t>(total, 1), 0u), pkj;
      bool kj_ok = true;
      const int wts = rows32_stride(nin);   // the row stride of the FP32 row kernel's term sums
      for (int t = 0; t < E.nedges; ++t) kj_ok = kj_ok && (long long)he.k[t] * wts + he.j[t] < (1 << 24);
      if (kj_ok) pkj.assign(packed.size(), 0u);
      for (int sl = 0; sl < E.nout; ++sl) {
        const int l = perm[sl];
        for (int t = he.ptr[l]; t < he.ptr[l + 1]; ++t) {
          const unsigned c = (unsigned)cls.at(he.c[t]);
          packed[tb[sl] + 32 * (t - he.ptr[l])] = ((unsigned)pair[t] << 8) | c;
          if (kj_ok) pkj[tb[sl] + 32 * (t - he.ptr[l])] = (c << 24) | (unsigned)(he.k[t] * wts + he.j[t]);
        }
      }
      if (E.nout < 65536) {
        // per slot: its first word and (output << 16 | couplings of the
        // warp's longest slot, the others padded with zero words), so the
        // lanes of a warp run the same coupling loop
        std::vector<int2> sd(E.nout);
        bool ok = true;
        for (int sl = 0; sl < E.nout; ++sl) {
          const int l = perm[sl], l0 = perm[sl & ~31];
          const int cnt = he.ptr[l0 + 1] - he.ptr[l0];
          ok = ok && cnt < 65536;
          sd[sl] = make_int2(tb[sl], (int)(((unsigned)l << 16) | (unsigned)cnt));
        }
        if (ok) {
          SG_TRY(upload(&E.sdesc, sd.data(), sd.size()));
          if (kj_ok) SG_TRY(upload(&E.ckj, pkj.data(), pkj.size()));
        }
      }
      df64* dt = nullptr;
      SG_TRY(upload(&E.ctr, packed.data(), packed.size()));
      SG_TRY(upload(&dt, tab.data(), tab.size()));
      E.ctab = dt;
      E.ncls = (int)tab.size();
    }
  }
  SG_TRY(upload(&E.pk, pk.data(), pk.size()));
  SG_TRY(upload(&E.pj, pj.data(), pj.size()));
  SG_TRY(upload(&E.pair, pair.data(), pair.size()));
  return SG_OK;
}

static void free_edges(EdgeList& E) {
  cudaFree(E.perm);
  cudaFree(E.ptr);
  cudaFree(E.k);
  cudaFree(E.j);
  cudaFree(E.c64);
  cudaFree(E.c32);
  cudaFree(E.cdf);
  cudaFree(E.ctr);
  cudaFree(E.ckj);
  cudaFree(E.sdesc);
  cudaFree(E.ctab);
  cudaFree(E.ctab32);
  cudaFree(E.pk);
  cudaFree(E.pj);
  cudaFree(E.pair);
  E = EdgeList();
}

// E[psi_a psi_b psi_c] of normalised 1-D Hermite polynomials: with s = (a+b+c)/2,
// sqrt(a! b! c!) / ((s-a)! (s-b)! (s-c)!) when s is an integer >= a, b, c, else 0.
static double hermite_triple(int a, int b, int c) {
  const int t = a + b + c;
  if (t & 1) return 0.0;
  const int s = t / 2;
  if (s < a || s < b || s < c) return 0.0;
  return std::exp(0.5 * (std::lgamma(a + 1.0) + std::lgamma(b + 1.0) + std::lgamma(c + 1.0)) -
                  std::lgamma(s - a + 1.0) - std::lgamma(s - b + 1.0) - std::lgamma(s - c + 1.0));
}

// Couplings of a gPC-expanded coefficient (Remark K-L): for every output l of
// [lo_out, hi_out) and input j of [lo_in, hi_in), every coefficient term
// i >= 1 with c = E[psi_i psi_j psi_l] != 0 (the product of the 1-D Hermite
// triple products over the coordinates). The term i = 0 is the identity
// (E[psi_j psi_l] = delta_jl): the diagonal part of the product kernels.
static HostEdges build_edges_gpc(const sg_problem* h, int lo_out, int hi_out, int lo_in, int hi_in) {
  HostEdges he;
  const int M = h->M;
  for (int l = lo_out; l < hi_out; ++l) {
    const int* al = h->alpha.data() + (size_t)l * M;
    for (int j = lo_in; j < hi_in; ++j) {
      const int* aj = h->alpha.data() + (size_t)j * M;
      for (int i = 1; i < h->nterm; ++i) {
        const int* gi = h->gamma.data() + (size_t)i * M;
        double c = 1.0;
        for (int k = 0; k < M && c != 0.0; ++k) c *= hermite_triple(gi[k], aj[k], al[k]);
        if (c == 0.0) continue;
        he.k.push_back(i);
        he.j.push_back(j - lo_in);
        he.c.push_back(c);
      }
    }
    he.ptr.push_back((int)he.k.size());
  }
  return he;
}

// Build the gather-form couplings. For every output column l of [lo_out, hi_out)
// and every KL index k, the neighbours alpha_l +- e_k inside [lo_in, hi_in).
static HostEdges build_edges(const sg_problem* h, const std::map<std::vector<int>, int>& index, int lo_out,
                             int hi_out, int lo_in, int hi_in) {
  HostEdges he;
  const int M = h->M;
  std::vector<int> b(M);
  for (int l = lo_out; l < hi_out; ++l) {
    const int* a = h->alpha.data() + (size_t)l * M;
    for (int k = 0; k < M; ++k) {
      for (int step = -1; step <= 1; step += 2) {
        for (int i = 0; i < M; ++i) b[i] = a[i];
        b[k] += step;
        if (b[k] < 0) continue;
        auto it = index.find(b);
        if (it == index.end()) continue;
        int j = it->second;
        if (j < lo_in || j >= hi_in) continue;
        he.k.push_back(k + 1);
        he.j.push_back(j - lo_in);
        he.c.push_back(xi_coupling(std::min(a[k], b[k]), h->family));
      }
    }
    he.ptr.push_back((int)he.k.size());
  }
  return he;
}

// Bilinear prolongation weight of coarse node X (fine position 2X+1) at fine node x.
static inline double w1(int d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); }

// Galerkin coarse stencil P^T A P for full coarsening with bilinear P.
static void galerkin_coarsen(int nx, int ny, const std::vector<double>& st, int nxc, int nyc,
                             std::vector<double>& stc) {
  stc.assign((size_t)nxc * nyc * 9, 0.0);
  for (int Y = 0; Y < nyc; ++Y) {
    for (int X = 0; X < nxc; ++X) {
      const size_t C = (size_t)Y * nxc + X;
      const int cxf = 2 * X + 1, cyf = 2 * Y + 1;
      for (int fy = cyf - 1; fy <= cyf + 1; ++fy) {
        for (int fx = cxf - 1; fx <= cxf + 1; ++fx) {
          const double wf = w1(fx - cxf) * w1(fy - cyf);
          const size_t f = (size_t)fy * nx + fx;
          for (int s = 0; s < 9; ++s) {
            const double a = st[f * 9 + s];
            if (a == 0.0) continue;
            const int gx = fx + (s % 3 - 1), gy = fy + (s / 3 - 1);
            int Xs[2], Ys[2];
            double wx[2], wy[2];
            int nxs = 0, nys = 0;
            if (gx & 1) { Xs[nxs] = (gx - 1) / 2; wx[nxs++] = 1.0; }
            else { Xs[nxs] = gx / 2 - 1; wx[nxs++] = 0.5; Xs[nxs] = gx / 2; wx[nxs++] = 0.5; }
            if (gy & 1) { Ys[nys] = (gy - 1) / 2; wy[nys++] = 1.0; }
            else { Ys[nys] = gy / 2 - 1; wy[nys++] = 0.5; Ys[nys] = gy / 2; wy[nys++] = 0.5; }
            for (int iy = 0; iy < nys; ++iy) {
              if (Ys[iy] < 0 || Ys[iy] >= nyc) continue;
              for (int ix = 0; ix < nxs; ++ix) {
                if (Xs[ix] < 0 || Xs[ix] >= nxc) continue;
                const int dX = Xs[ix] - X, dY = Ys[iy] - Y;
                stc[C * 9 + (dY + 1) * 3 + (dX + 1)] += wf * a * wx[ix] * wy[iy];
              }
            }
          }
        }
      }
    }
  }
}

static int upload_grid(GridLevel& g, const std::vector<double>& st) {
  SG_TRY(upload(&g.st_base, st.data(), st.size()));
  std::vector<float> st32(st.begin(), st.end());
  std::vector<double> dinv(g.n);
  for (int i = 0; i < g.n; ++i) dinv[i] = 1.0 / st[(size_t)i * 9 + 4];
  std::vector<float> dinv32(dinv.begin(), dinv.end());
  SG_TRY(upload(&g.st64, st.data(), st.size()));
  SG_TRY(upload(&g.st32, st32.data(), st32.size()));
  SG_TRY(upload(&g.dinv64, dinv.data(), dinv.size()));
  SG_TRY(upload(&g.dinv32, dinv32.data(), dinv32.size()));
  return SG_OK;
}

static int setup_impl(const sg_mesh* mesh, int M, int p, int family, int n, int nnz, const int* rowptr,
                      const int* colidx, const double* vals, const double* mass_vals, sg_problem* h, int q) {
  if (q >= 0 && (family != SG_HERMITE || M < 1 || q > 16)) {
    set_error("sg_setup_gpc: the gPC coefficient needs Hermite chaos, M >= 1 and a degree q <= 16");
    return q >= 0 && family != SG_HERMITE ? SG_ERR_UNSUPPORTED : SG_ERR_INVALID_ARG;
  }
  if (M < 0 || p < 0 || n <= 0 || nnz <= 0 || !rowptr || !colidx || !vals) {
    set_error("sg_setup: invalid sizes or null pointers (M=%d p=%d n=%d nnz=%d)", M, p, n, nnz);
    return SG_ERR_INVALID_ARG;
  }
  if (family != SG_LEGENDRE && family != SG_HERMITE) {
    set_error("sg_setup: unknown chaos family %d", family);
    return SG_ERR_INVALID_ARG;
  }
  if (rowptr[0] != 0 || rowptr[n] != nnz) {
    set_error("sg_setup: rowptr[0] must be 0 and rowptr[n] == nnz");
    return SG_ERR_INVALID_ARG;
  }
  int max_row = 0;
  for (int r = 0; r < n; ++r) {
    if (rowptr[r + 1] < rowptr[r]) {
      set_error("sg_setup: rowptr not monotone at row %d", r);
      return SG_ERR_INVALID_ARG;
    }
    max_row = std::max(max_row, rowptr[r + 1] - rowptr[r]);
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      if (colidx[e] < 0 || colidx[e] >= n || (e > rowptr[r] && colidx[e] <= colidx[e - 1])) {
        set_error("sg_setup: column index out of range or unsorted in row %d", r);
        return SG_ERR_INVALID_ARG;
      }
    }
  }
  // value terms per nonzero: the linear KL expansion has M + 1, the gPC one C(M + q, M)
  long long nterm = M + 1;
  if (q >= 0) {
    nterm = 1;
    for (int i = 1; i <= M; ++i) nterm = nterm * (q + i) / i;
    if (nterm > 4096) {
      set_error("sg_setup_gpc: %lld coefficient terms exceed the supported 4096", nterm);
      return SG_ERR_UNSUPPORTED;
    }
  }
  h->q = q;
  h->nterm = (int)nterm;
  const size_t nv = (size_t)nnz * nterm;
  for (size_t i = 0; i < nv; ++i) {
    if (!std::isfinite(vals[i])) {
      set_error("sg_setup: non-finite matrix value at %zu", i);
      return SG_ERR_INVALID_ARG;
    }
  }
  h->n = n;
  h->nnz = nnz;
  h->M = M;
  h->p = p;
  h->family = family;
  h->max_row_nnz = max_row;
  SG_TRY_CUDA(cudaGetDevice(&h->device));
  SG_TRY_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  SG_TRY_CUDA(cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));

  // chaos table
  h->off.assign(1, 0);
  std::vector<int> cur(std::max(M, 1));
  for (int d = 0; d <= p; ++d) {
    if (M == 0) {  // the constant polynomial only
      h->off.push_back(1);
      continue;
    }
    emit_degree(M, 0, d, cur, h->alpha);
    h->off.push_back((int)(h->alpha.size() / M));
  }
  h->P = h->off.back();
  if (M == 0) h->alpha.clear();
  h->wmax = 0;
  for (int d = 0; d <= p; ++d) h->wmax = std::max(h->wmax, h->off[d + 1] - h->off[d]);
  if (h->P > 2048) {
    set_error("sg_setup: P = %d chaos polynomials exceeds the supported 2048", h->P);
    return SG_ERR_UNSUPPORTED;
  }

  std::map<std::vector<int>, int> index;
  for (int l = 0; l < h->P; ++l)
    index[std::vector<int>(h->alpha.begin() + (size_t)l * M, h->alpha.begin() + (size_t)(l + 1) * M)] = l;
  const std::vector<int>& off = h->off;
  h->pre.resize(p + 1);
  h->post.resize(p + 1);
  if (q < 0) {
    SG_TRY(upload_edges(build_edges(h, index, 0, h->P, 0, h->P), h->all, 0, 0, h->P));
    for (int l = 1; l <= p; ++l) {
      SG_TRY(upload_edges(build_edges(h, index, off[l - 1], off[l], off[l], off[l + 1]), h->pre[l], off[l - 1],
                          off[l], off[l + 1] - off[l]));
      SG_TRY(upload_edges(build_edges(h, index, off[l], off[l + 1], off[l - 1], off[l]), h->post[l], off[l],
                          off[l - 1], off[l] - off[l - 1]));
    }
    if (p >= 1) SG_TRY(upload_edges(build_edges(h, index, 0, off[p], 0, off[p]), h->sub, 0, 0, off[p]));
  } else {
    // the coefficient terms in the same graded order
    std::vector<int> cur(M);
    for (int d = 0; d <= q; ++d) emit_degree(M, 0, d, cur, h->gamma);
    SG_TRY(upload_edges(build_edges_gpc(h, 0, h->P, 0, h->P), h->all, 0, 0, h->P));
    h->dlev.resize(p + 1);
    for (int l = 1; l <= p; ++l) {
      // B_l: every lower level from level l; C_l: level l from every lower level; D_l: level l with itself
      SG_TRY(upload_edges(build_edges_gpc(h, 0, off[l], off[l], off[l + 1]), h->pre[l], 0, off[l],
                          off[l + 1] - off[l]));
      SG_TRY(upload_edges(build_edges_gpc(h, off[l], off[l + 1], 0, off[l]), h->post[l], off[l], 0, off[l]));
      SG_TRY(upload_edges(build_edges_gpc(h, off[l], off[l + 1], off[l], off[l + 1]), h->dlev[l], off[l], off[l],
                          off[l + 1] - off[l]));
    }
    // the pair form keeps one sum per distinct (term, input) in shared memory:
    // too many with a dense coupling, so the gPC products use the gather form
    h->k1_pairs[0] = h->k1_pairs[1] = h->outer_pairs = 0;
  }

  // matrices
  SG_TRY(upload(&h->rowptr, rowptr, (size_t)n + 1));
  SG_TRY(upload(&h->colidx, colidx, (size_t)nnz));
  SG_TRY(upload(&h->vals64, vals, nv));
  SG_TRY(upload(&h->vals_base, vals, nv));
  h->scales.assign(h->nterm, 1.0);
  SG_TRY(upload(&h->scales_dev, h->scales.data(), h->scales.size()));
  {
    std::vector<float> v32(vals, vals + nv);
    SG_TRY(upload(&h->vals32, v32.data(), nv));
    std::vector<df64> vdf(nv);
    for (size_t i = 0; i < nv; ++i) vdf[i] = df_split_host(vals[i]);
    df64* d = nullptr;
    SG_TRY(upload(&d, vdf.data(), nv));
    h->vals_df = d;
  }
  if (mass_vals) SG_TRY(upload(&h->mass64, mass_vals, (size_t)nnz));

  // multigrid hierarchy of A_0 on the structured grid
  if (mesh && mesh->ne_x > 1 && mesh->ne_y > 1) {
    const int nx = mesh->ne_x - 1, ny = mesh->ne_y - 1;
    if ((long long)nx * ny != n) {
      set_error("sg_setup: mesh %dx%d has %d interior nodes, n = %d", mesh->ne_x, mesh->ne_y, nx * ny, n);
      return SG_ERR_INVALID_ARG;
    }
    const int ne = mesh->ne_x;
    // the inner solves need the 9-point stencil of A_0 on the grid; the
    // multigrid hierarchy also a power-of-two square mesh
    const bool pow2 = mesh->ne_x == mesh->ne_y && (ne & (ne - 1)) == 0;
    bool ok = true;
    std::vector<double> st((size_t)n * 9, 0.0);
    for (int r = 0; r < n && ok; ++r) {
      const int x = r % nx, y = r / nx;
      for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const int c = colidx[e], cx = c % nx, cy = c / nx;
        const int dx = cx - x, dy = cy - y;
        if (dx < -1 || dx > 1 || dy < -1 || dy > 1) { ok = false; break; }
        st[(size_t)r * 9 + (dy + 1) * 3 + (dx + 1)] += vals[(size_t)e * h->nterm];
      }
      if (ok && !(st[(size_t)r * 9 + 4] > 0.0)) ok = false;
    }
    if (ok) {
      h->nx = nx;
      h->ny = ny;
      int gx = nx, gy = ny;
      while (true) {
        GridLevel g;
        g.nx = gx; g.ny = gy; g.n = gx * gy;
        SG_TRY(upload_grid(g, st));
        h->grids.push_back(g);
        if (!pow2) break;            // the finest grid alone: diagonal M_0 only
        if (gx <= 1) {
          h->mg_full = true;
          break;
        }
        const int nxc = (gx - 1) / 2, nyc = (gy - 1) / 2;
        std::vector<double> stc;
        galerkin_coarsen(gx, gy, st, nxc, nyc, stc);
        st.swap(stc);
        gx = nxc; gy = nyc;
      }
    }
  }
  // the in-block coarse V-cycle takes over at the first grid with <= 1024 nodes
  h->cb_level = (int)h->grids.size();
  for (int g = 0; g < (int)h->grids.size(); ++g)
    if (h->grids[g].n <= 1024) { h->cb_level = g; break; }
  if (h->mg_full) SG_TRY(cluster_setup(h));
  for (auto& cs : h->cap) SG_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  {
    const char* ev = getenv("SGHSC_EAGER");
    h->eager = ev && ev[0] == '1';
  }
  {
    const char* ev = getenv("SGHSC_NO_PIPE");
    h->pipe_off = ev && ev[0] == '1';
  }
  {
    const char* ev = getenv("SGHSC_GATHER_FORM");   // start from the gather form of the full product
    if (ev && ev[0] == '1') h->k1_pairs[0] = h->k1_pairs[1] = h->outer_pairs = h->outer_pairs_df = 0;
    const char* eg = getenv("SGHSC_GENERIC_PRODUCTS");   // the one-row-at-a-time kernels only
    if ((ev && ev[0] == '1') || (eg && eg[0] == '1')) h->staged_pairs = 0;
  }
  SG_TRY_CUDA(cudaMalloc((void**)&h->loopflags, 8 * sizeof(int)));
  SG_TRY_CUDA(cudaMemset(h->loopflags, 0, 8 * sizeof(int)));
  SG_TRY_CUDA(cudaMallocHost((void**)&h->loopflag_host, sizeof(int)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->status, sizeof(int)));
  SG_TRY_CUDA(cudaMemset(h->status, 0, sizeof(int)));
  SG_TRY_CUDA(cudaMallocHost((void**)&h->status_host, sizeof(int)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->iacc, 2 * sizeof(long long)));
  SG_TRY_CUDA(cudaMemset(h->iacc, 0, 2 * sizeof(long long)));
  return SG_OK;
}

// vals = base * scale[k] for every nonzero (FP64 and FP32 copies)
__global__ void k_scale_vals(long long count, int M1, const double* __restrict__ base, const double* __restrict__ scale,
                             double* __restrict__ v64, float* __restrict__ v32, df64* __restrict__ vdf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const double v = base[i] * scale[i % M1];
    v64[i] = v;
    v32[i] = (float)v;
    const float h = __double2float_rn(v);
    vdf[i] = df64(h, __double2float_rn(v - (double)h));
  }
}

// multigrid stencils of s * A_0: st = s * base, dinv = 1 / (s * base_centre)
__global__ void k_scale_grid(int n, const double* __restrict__ base, double s, double* __restrict__ st64,
                             float* __restrict__ st32, double* __restrict__ dinv64, float* __restrict__ dinv32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 9; i += gridDim.x * blockDim.x) {
    const double v = s * base[i];
    st64[i] = v;
    st32[i] = (float)v;
    if (i % 9 == 4) {
      dinv64[i / 9] = 1.0 / v;
      dinv32[i / 9] = (float)(1.0 / v);
    }
  }
}

}  // namespace sghsc

using namespace sghsc;

extern "C" {

int sg_set_scales(sg_problem* h, const double* scale) {
  set_error("");
  if (!h || !scale) {
    set_error("sg_set_scales: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  for (int k = 0; k < h->nterm; ++k)
    if (!std::isfinite(scale[k])) {
      set_error("sg_set_scales: non-finite scale %d", k);
      return SG_ERR_INVALID_ARG;
    }
  if (!(scale[0] > 0.0) && !h->grids.empty()) {
    set_error("sg_set_scales: the mean matrix needs a positive scale");
    return SG_ERR_INVALID_ARG;
  }
  SG_TRY_CUDA(cudaDeviceSynchronize());   // no solve may be reading the values
  h->scales.assign(scale, scale + h->nterm);
  SG_TRY_CUDA(cudaMemcpy(h->scales_dev, scale, h->nterm * sizeof(double), cudaMemcpyHostToDevice));
  const long long count = (long long)h->nnz * h->nterm;
  { k_scale_vals<<<(int)std::min<long long>((count + 255) / 256, 4096), 256>>>(count, h->nterm, h->vals_base, h->scales_dev, h->vals64, h->vals32, (df64*)h->vals_df); ::sghsc::note_launch(); }
  for (auto& g : h->grids)
    { k_scale_grid<<<std::min((g.n * 9 + 255) / 256, 4096), 256>>>(g.n, g.st_base, scale[0], g.st64, g.st32, g.dinv64, g.dinv32); ::sghsc::note_launch(); }
  SG_TRY_CUDA(cudaGetLastError());
  SG_TRY_CUDA(cudaDeviceSynchronize());
  return SG_OK;
}


const char* sg_last_error(void) { return sghsc::g_err; }

long long sg_kernel_launches(void) { return sghsc::g_launches.load(); }

void sg_default_prec_opts(sg_prec_opts* o) {
  if (!o) return;
  o->precision = SG_F32;
  o->top_level_f64 = 1;
  o->inner_tol = 1e-2;
  o->inner_maxit = 200;
  o->inner_fixed_iters = 0;
  o->nu = 2;
  o->omega = 0.8;
  o->m0 = SG_M0_VCYCLE;
  o->level_tol = 1e-8;
  o->level_maxit = 500;
  o->md_m0 = 0;
  o->df64 = 0;
}

void sg_default_solve_opts(sg_solve_opts* o) {
  if (!o) return;
  o->precond = SG_PREC_HSC;
  sg_default_prec_opts(&o->prec);
  o->tol = 1e-8;
  o->maxit = 500;
  o->flexible = 1;
  o->use_x0 = 0;
  o->check_true_residual = 1;
  o->schur_reduced = 0;
  o->schur_inner_tol = 1e-11;
}

int sg_setup(const sg_mesh* mesh, int M, int p, int family, int n, int nnz, const int* rowptr,
             const int* colidx, const double* vals, const double* mass_vals, sg_problem** out) {
  set_error("");
  if (!out) {
    set_error("sg_setup: out is null");
    return SG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sg_problem* h = new sg_problem();
  int st = setup_impl(mesh, M, p, family, n, nnz, rowptr, colidx, vals, mass_vals, h, -1);
  if (st != SG_OK) {
    sg_destroy(h);
    return st;
  }
  *out = h;
  return SG_OK;
}

int sg_setup_gpc(const sg_mesh* mesh, int M, int p, int q, int family, int n, int nnz, const int* rowptr,
                 const int* colidx, const double* vals, const double* mass_vals, sg_problem** out) {
  set_error("");
  if (!out) {
    set_error("sg_setup_gpc: out is null");
    return SG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (q < 0) {
    set_error("sg_setup_gpc: q < 0");
    return SG_ERR_INVALID_ARG;
  }
  sg_problem* h = new sg_problem();
  int st = setup_impl(mesh, M, p, family, n, nnz, rowptr, colidx, vals, mass_vals, h, q);
  if (st != SG_OK) {
    sg_destroy(h);
    return st;
  }
  *out = h;
  return SG_OK;
}

int sg_problem_terms(const sg_problem* h, int* nterm, int* q) {
  if (!h) {
    set_error("sg_problem_terms: null handle");
    return SG_ERR_INVALID_ARG;
  }
  if (nterm) *nterm = h->nterm;
  if (q) *q = h->q;
  return SG_OK;
}

void sg_destroy(sg_problem* h) {
  if (!h) return;
  free_edges(h->all);
  for (auto& e : h->pre) free_edges(e);
  for (auto& e : h->post) free_edges(e);
  free_edges(h->sub);
  for (auto& e : h->dlev) free_edges(e);
  for (auto& g : h->grids) {
    cudaFree(g.st_base); cudaFree(g.st64); cudaFree(g.st32); cudaFree(g.dinv64); cudaFree(g.dinv32);
  }
  if (h->cap[0]) cudaDeviceSynchronize();
  clear_graphs(h);
  free_inner_work(h);
  cluster_free(h);
  void* bufs[] = {h->rowptr, h->colidx, h->vals64, h->vals32, h->mass64, h->R32, h->Z32, h->T32, h->R64w,
                  h->T64, h->fF, h->fx, h->fr, h->fz, h->fpA, h->fpB, h->fq, h->opart, h->osc, h->octl,
                  h->hist_alpha, h->hist_beta, h->hist_res, h->io_in, h->io_out, h->status, h->iacc, h->wdev, h->loopflags, h->vals_base, h->scales_dev, h->fG, h->vals_df,
                  h->lx, h->lr, h->lz, h->lp, h->lq, h->lb, h->lctl, h->lsc, h->lhist_alpha, h->lhist_beta,
                  h->lhist_res};
  for (void* b : bufs) cudaFree(b);
  for (auto& cs : h->cap)
    if (cs) cudaStreamDestroy(cs);
  if (h->osc_host) cudaFreeHost(h->osc_host);
  if (h->status_host) cudaFreeHost(h->status_host);
  if (h->loopflag_host) cudaFreeHost(h->loopflag_host);
  delete h;
}

int sg_problem_dims(const sg_problem* h, int* n, int* P, int* M, int* p, int* nnz) {
  if (!h) {
    set_error("sg_problem_dims: null handle");
    return SG_ERR_INVALID_ARG;
  }
  if (n) *n = h->n;
  if (P) *P = h->P;
  if (M) *M = h->M;
  if (p) *p = h->p;
  if (nnz) *nnz = h->nnz;
  return SG_OK;
}

int sg_chaos_table(const sg_problem* h, int* alpha, int* level_offsets) {
  if (!h) {
    set_error("sg_chaos_table: null handle");
    return SG_ERR_INVALID_ARG;
  }
  if (alpha && !h->alpha.empty()) std::memcpy(alpha, h->alpha.data(), h->alpha.size() * sizeof(int));
  if (level_offsets) std::memcpy(level_offsets, h->off.data(), h->off.size() * sizeof(int));
  return SG_OK;
}

}  // extern "C"
