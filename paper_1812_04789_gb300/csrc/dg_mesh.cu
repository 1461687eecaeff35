// Mesh handle: periodic structured mesh, orthonormal total-degree Legendre
// basis, Gauss-Legendre quadrature and the BR2 lifting operator, built on the
// host in FP64 and uploaded in FP64 and FP32 (Sec. 3, eq. BSpace; Sec. 3.1).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "dg_internal.h"

namespace dgk {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 0) ? 1.0 : p1;
      double pm = (n == 0) ? 0.0 : p0;
      double dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        // final derivative at the converged node
        p0 = 1.0;
        p1 = z;
        for (int k = 1; k < n; ++k) {
          double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
    }
  }
  if (n == 1) {
    x[0] = 0.0;
    w[0] = 2.0;
  }
}

// Orthonormal Legendre Lt_k = sqrt((2k+1)/2) P_k and derivative at z.
static void legendre(int pmax, double z, double* L, double* dL) {
  std::vector<double> P(pmax + 2), dP(pmax + 2);
  P[0] = 1.0;
  dP[0] = 0.0;
  if (pmax >= 1) {
    P[1] = z;
    dP[1] = 1.0;
  }
  for (int k = 1; k < pmax; ++k) {
    P[k + 1] = ((2.0 * k + 1.0) * z * P[k] - k * P[k - 1]) / (k + 1.0);
    dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
  }
  for (int k = 0; k <= pmax; ++k) {
    double s = sqrt((2.0 * k + 1.0) / 2.0);
    L[k] = s * P[k];
    dL[k] = s * dP[k];
  }
}

// Total-degree multi-indices ordered by degree, then lexicographically with
// the first index descending.
static std::vector<std::array<int, 3>> mode_list(int p, int d, int space) {
  std::vector<std::array<int, 3>> out;
  if (space == DG_SPACE_Q) {   // largest 1-D degree s, then descending lexicographic
    for (int s = 0; s <= p; ++s)
      for (int a = s; a >= 0; --a)
        for (int b = s; b >= 0; --b)
          for (int c = (d == 3 ? s : 0); c >= 0; --c)
            if (std::max(a, std::max(b, c)) == s) out.push_back({a, b, d == 3 ? c : 0});
    return out;
  }
  for (int s = 0; s <= p; ++s) {
    std::vector<std::array<int, 3>> lv;
    for (int a = s; a >= 0; --a) {
      if (d == 2) {
        lv.push_back({a, s - a, 0});
      } else {
        for (int b = s - a; b >= 0; --b) lv.push_back({a, b, s - a - b});
      }
    }
    out.insert(out.end(), lv.begin(), lv.end());
  }
  return out;
}

template <class T>
static cudaError_t upload(Mesh& M, const std::vector<double>& h, T** dst) {
  std::vector<T> tmp(h.size());
  for (size_t i = 0; i < h.size(); ++i) tmp[i] = (T)h[i];
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(1, h.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  M.allocs.push_back(*dst);
  return cudaMemcpy(*dst, tmp.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <class T>
static cudaError_t upload_tables(Mesh& M, Tables<T>& t, const std::vector<double>* tabs) {
  cudaError_t e;
  T** dst[14] = {&t.vphiT, &t.vdphiT, &t.vphi, &t.vdphi, &t.vw, &t.fphiT, &t.fdphiT,
                 &t.fphi,  &t.fdphi,  &t.fw,   &t.lift,  &t.liftT, &t.fpk, &t.fpw};
  for (int i = 0; i < 14; ++i)
    if ((e = upload<T>(M, tabs[i], dst[i])) != cudaSuccess) return e;
  size_t ns = (size_t)M.E * M.d * 2 * M.nb;
  if ((e = cudaMalloc((void**)&t.slots, ns * sizeof(T))) != cudaSuccess) return e;
  M.allocs.push_back(t.slots);
  size_t nd = (size_t)M.E * M.nb;
  if ((e = cudaMalloc((void**)&t.fd_w, nd * sizeof(T))) != cudaSuccess) return e;
  M.allocs.push_back(t.fd_w);
  if ((e = cudaMalloc((void**)&t.fd_r, nd * sizeof(T))) != cudaSuccess) return e;
  M.allocs.push_back(t.fd_r);
  if ((e = cudaMalloc((void**)&t.fd_o, nd * sizeof(T))) != cudaSuccess) return e;
  M.allocs.push_back(t.fd_o);
  return cudaSuccess;
}

void free_mesh(Mesh& M) {
  for (void* p : M.allocs) cudaFree(p);
  M.allocs.clear();
}

template <>
MeshView<double> Mesh::view<double>() const {
  MeshView<double> v;
  v.d = d; v.m = m; v.nm = nm; v.nb = nb; v.nq = nq; v.nqf = nqf; v.E = E;
  for (int k = 0; k < 3; ++k) v.n[k] = desc.n[k];
  v.nbr = nbr;
  v.vphiT = t64.vphiT; v.vdphiT = t64.vdphiT; v.vphi = t64.vphi; v.vdphi = t64.vdphi; v.vw = t64.vw;
  v.fphiT = t64.fphiT; v.fdphiT = t64.fdphiT; v.fphi = t64.fphi; v.fdphi = t64.fdphi; v.fw = t64.fw;
  v.lift = t64.lift;
  v.liftT = t64.liftT;
  v.fpk = t64.fpk;
  v.fpw = t64.fpw;
  v.detJ = detJ;
  return v;
}
template <>
MeshView<float> Mesh::view<float>() const {
  MeshView<float> v;
  v.d = d; v.m = m; v.nm = nm; v.nb = nb; v.nq = nq; v.nqf = nqf; v.E = E;
  for (int k = 0; k < 3; ++k) v.n[k] = desc.n[k];
  v.nbr = nbr;
  v.vphiT = t32.vphiT; v.vdphiT = t32.vdphiT; v.vphi = t32.vphi; v.vdphi = t32.vdphi; v.vw = t32.vw;
  v.fphiT = t32.fphiT; v.fdphiT = t32.fdphiT; v.fphi = t32.fphi; v.fdphi = t32.fdphi; v.fw = t32.fw;
  v.lift = t32.lift;
  v.liftT = t32.liftT;
  v.fpk = t32.fpk;
  v.fpw = t32.fpw;
  v.detJ = (float)detJ;
  return v;
}
template <class T>
Phys<T> Mesh::phys_t() const {
  Phys<T> p;
  p.gamma = (T)phys.gamma;
  p.gm1 = (T)(phys.gamma - 1.0);
  p.Pr = (T)phys.Pr;
  p.mu = (T)phys.mu;
  p.Rgas = (T)phys.Rgas;
  p.eta = (T)(phys.eta_br2 > 0 ? phys.eta_br2 : 2.0 * d + 1.0);
  p.roe_delta = (T)phys.roe_delta;
  p.kappa = (T)(phys.mu * phys.gamma * phys.Rgas / ((phys.gamma - 1.0) * phys.Pr));
  return p;
}
template Phys<double> Mesh::phys_t<double>() const;
template Phys<float> Mesh::phys_t<float>() const;

static dg_status build_mesh(Mesh& M, const dg_mesh_desc* desc, const dg_physics* ph) {
  M.desc = *desc;
  M.phys = *ph;
  M.d = desc->dim;
  M.m = M.d + 2;
  M.p = desc->p;
  M.nq1d = desc->nq1d > 0 ? desc->nq1d : desc->p + 2;
  const int d = M.d, p = M.p, nq1 = M.nq1d;
  auto modes = mode_list(p, d, desc->space);
  M.nm = (int)modes.size();
  M.nb = M.m * M.nm;
  M.nq = 1;
  for (int k = 0; k < d; ++k) M.nq *= nq1;
  M.nqf = M.nq / nq1;
  M.E = 1;
  for (int k = 0; k < d; ++k) M.E *= desc->n[k];
  M.detJ = 1.0;
  double metric[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    M.h[k] = (desc->hi[k] - desc->lo[k]) / desc->n[k];
    M.detJ *= M.h[k] / 2.0;
    metric[k] = 2.0 / M.h[k];
  }
  for (int k = 0; k < d; ++k) {
    M.faceJ[k] = 1.0;
    for (int kk = 0; kk < d; ++kk)
      if (kk != k) M.faceJ[k] *= M.h[kk] / 2.0;
  }
  std::vector<double> xg, wg;
  gauss_legendre(nq1, xg, wg);
  // 1-D tables at the GL points and at the end points -1, +1
  std::vector<double> L((size_t)nq1 * (p + 1)), dL((size_t)nq1 * (p + 1));
  for (int a = 0; a < nq1; ++a) legendre(p, xg[a], &L[(size_t)a * (p + 1)], &dL[(size_t)a * (p + 1)]);
  std::vector<double> Le(2 * (p + 1)), dLe(2 * (p + 1));
  legendre(p, -1.0, &Le[0], &dLe[0]);
  legendre(p, 1.0, &Le[p + 1], &dLe[p + 1]);
  auto L1 = [&](int a, int deg) { return L[(size_t)a * (p + 1) + deg]; };
  auto dL1 = [&](int a, int deg) { return dL[(size_t)a * (p + 1) + deg]; };

  const int nq = M.nq, nqf = M.nqf, nm = M.nm;
  std::vector<double> tabs[14];
  std::vector<double>&vphiT = tabs[0], &vdphiT = tabs[1], &vphi = tabs[2], &vdphi = tabs[3], &vw = tabs[4];
  std::vector<double>&fphiT = tabs[5], &fdphiT = tabs[6], &fphi = tabs[7], &fdphi = tabs[8], &fw = tabs[9];
  std::vector<double>& lift = tabs[10];
  std::vector<double>& liftT = tabs[11];
  vphiT.assign((size_t)nm * nq, 0);
  vdphiT.assign((size_t)d * nm * nq, 0);
  vphi.assign((size_t)nq * nm, 0);
  vdphi.assign((size_t)d * nq * nm, 0);
  vw.assign(nq, 0);
  for (int q = 0; q < nq; ++q) {
    int a[3] = {0, 0, 0};
    int r = q;
    for (int k = 0; k < d; ++k) {
      a[k] = r % nq1;
      r /= nq1;
    }
    double w = M.detJ;
    for (int k = 0; k < d; ++k) w *= wg[a[k]];
    vw[q] = w;
    for (int i = 0; i < nm; ++i) {
      double val = 1.0;
      for (int k = 0; k < d; ++k) val *= L1(a[k], modes[i][k]);
      vphi[(size_t)q * nm + i] = val;
      vphiT[(size_t)i * nq + q] = val;
      for (int kk = 0; kk < d; ++kk) {
        double g = metric[kk];
        for (int k = 0; k < d; ++k) g *= (k == kk) ? dL1(a[k], modes[i][k]) : L1(a[k], modes[i][k]);
        vdphi[((size_t)kk * nq + q) * nm + i] = g;
        vdphiT[((size_t)kk * nm + i) * nq + q] = g;
      }
    }
  }
  // faces: local face f = 2k + side, side 0 at xi_k = -1, side 1 at xi_k = +1;
  // face points run over the other coordinates in increasing order, first fastest
  const int nf = 2 * d;
  fphiT.assign((size_t)nf * nm * nqf, 0);
  fdphiT.assign((size_t)nf * d * nm * nqf, 0);
  fphi.assign((size_t)nf * nqf * nm, 0);
  fdphi.assign((size_t)nf * d * nqf * nm, 0);
  fw.assign((size_t)d * nqf, 0);
  lift.assign((size_t)nf * nqf * nqf, 0);
  std::vector<double> wraw(nqf);
  for (int f = 0; f < nf; ++f) {
    int k = f / 2, side = f % 2;
    int tang[2] = {0, 0}, nt = 0;
    for (int kk = 0; kk < d; ++kk)
      if (kk != k) tang[nt++] = kk;
    for (int q = 0; q < nqf; ++q) {
      int b[2] = {q % nq1, (nq1 > 0) ? q / nq1 : 0};
      double wr = 1.0;
      for (int t = 0; t < nt; ++t) wr *= wg[b[t]];
      wraw[q] = wr;
      if (side == 0) fw[(size_t)k * nqf + q] = wr * M.faceJ[k];
      for (int i = 0; i < nm; ++i) {
        double vals[3], ders[3];
        for (int kk = 0; kk < d; ++kk) {
          int deg = modes[i][kk];
          if (kk == k) {
            vals[kk] = Le[side * (p + 1) + deg];
            ders[kk] = dLe[side * (p + 1) + deg];
          } else {
            int t = (kk == tang[0]) ? 0 : 1;
            vals[kk] = L1(b[t], deg);
            ders[kk] = dL1(b[t], deg);
          }
        }
        double val = 1.0;
        for (int kk = 0; kk < d; ++kk) val *= vals[kk];
        fphi[((size_t)f * nqf + q) * nm + i] = val;
        fphiT[((size_t)f * nm + i) * nqf + q] = val;
        for (int kk = 0; kk < d; ++kk) {
          double g = metric[kk];
          for (int k3 = 0; k3 < d; ++k3) g *= (k3 == kk) ? ders[k3] : vals[k3];
          fdphi[(((size_t)f * d + kk) * nqf + q) * nm + i] = g;
          fdphiT[(((size_t)f * d + kk) * nm + i) * nqf + q] = g;
        }
      }
    }
    // BR2 lifting at face points (eq. re): delta(q) = |J_F|/(2|J|) sum_i phi_i(q)
    // sum_q' w_q' phi_i(q') X(q')  =>  P_f[q][q'] (mass matrix |J| I), stored by
    // columns, lift[f][q'][q]: a warp's points q of one column are consecutive
    double cl = M.faceJ[k] / (2.0 * M.detJ);
    for (int q = 0; q < nqf; ++q)
      for (int q2 = 0; q2 < nqf; ++q2) {
        double s = 0;
        for (int i = 0; i < nm; ++i)
          s += fphi[((size_t)f * nqf + q) * nm + i] * fphi[((size_t)f * nqf + q2) * nm + i];
        lift[((size_t)f * nqf + q2) * nqf + q] = cl * s * wraw[q2];
      }
  }
  // lifted test functions: the BR2 term sum_q fw(q) phi_i(q) {delta}(q) is linear
  // in the lifted tensors, so it equals sum_q' liftT[f][c][q'][i] G_c(q') with
  // liftT[f][c][q'][i] = sum_q fw(q) phi^f_i(q) P_c[q][q'], P_0 = lift of the face's
  // +k side (2k+1), P_1 = lift of its -k side (2k)
  liftT.assign((size_t)nf * 2 * nqf * nm, 0);
  for (int f = 0; f < nf; ++f) {
    int k = f / 2;
    for (int c = 0; c < 2; ++c) {
      int pf = c == 0 ? 2 * k + 1 : 2 * k;
      for (int q2 = 0; q2 < nqf; ++q2)
        for (int i = 0; i < nm; ++i) {
          double s = 0;
          for (int q = 0; q < nqf; ++q)
            s += fw[(size_t)k * nqf + q] * fphi[((size_t)f * nqf + q) * nm + i] *
                 lift[((size_t)pf * nqf + q2) * nqf + q];
          liftT[(((size_t)f * 2 + c) * nqf + q2) * nm + i] = s;
        }
    }
  }
  // packed traces for 16-byte loads: fpk[f][i][q] = (phi, grad phi) at point q,
  // fpw[f][q][i] = fw(q) (phi, grad phi)
  std::vector<double>&fpk = tabs[12], &fpw = tabs[13];
  fpk.assign((size_t)nf * nm * nqf * 4, 0);
  fpw.assign((size_t)nf * nqf * nm * 4, 0);
  for (int f = 0; f < nf; ++f)
    for (int q = 0; q < nqf; ++q) {
      const double wq = fw[(size_t)(f / 2) * nqf + q];
      for (int i = 0; i < nm; ++i) {
        double e[4] = {fphi[((size_t)f * nqf + q) * nm + i], 0, 0, 0};
        for (int kk = 0; kk < d; ++kk) e[1 + kk] = fdphi[(((size_t)f * d + kk) * nqf + q) * nm + i];
        for (int c = 0; c < 4; ++c) {
          fpk[(((size_t)f * nm + i) * nqf + q) * 4 + c] = e[c];
          fpw[(((size_t)f * nqf + q) * nm + i) * 4 + c] = wq * e[c];
        }
      }
    }
  // neighbours
  std::vector<int> nbr((size_t)M.E * d * 2);
  for (int e = 0; e < M.E; ++e) {
    int ijk[3] = {0, 0, 0}, r = e;
    for (int k = 0; k < d; ++k) {
      ijk[k] = r % desc->n[k];
      r /= desc->n[k];
    }
    for (int k = 0; k < d; ++k)
      for (int side = 0; side < 2; ++side) {
        int j[3] = {ijk[0], ijk[1], ijk[2]};
        j[k] = (j[k] + (side ? 1 : -1) + desc->n[k]) % desc->n[k];
        int idx = 0;
        for (int kk = d - 1; kk >= 0; --kk) idx = idx * desc->n[kk] + j[kk];
        nbr[((size_t)e * d + k) * 2 + side] = idx;
      }
  }
  cudaError_t err;
  if ((err = cudaMalloc((void**)&M.nbr, nbr.size() * sizeof(int))) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.nbr);
  if ((err = cudaMemcpy(M.nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
    return DG_ERR_CUDA;
  if ((err = upload_tables<double>(M, M.t64, tabs)) != cudaSuccess)
    return err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  if ((err = upload_tables<float>(M, M.t32, tabs)) != cudaSuccess)
    return err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  {   // one-dimensional factors for sum factorisation (Q_p, and P_p embedded in Q_p)
    const int n1 = p + 1;
    // layout: L[a][q], dL[a][q] (reference derivative), w[q], then the end
    // values L_a(-1), L_a(+1) and dL_a(-1), dL_a(+1) (face traces)
    std::vector<double> l1d((size_t)2 * n1 * nq1 + nq1 + 4 * n1);
    for (int a = 0; a < n1; ++a)
      for (int q = 0; q < nq1; ++q) {
        l1d[(size_t)a * nq1 + q] = L1(q, a);
        l1d[(size_t)(n1 + a) * nq1 + q] = dL1(q, a);
      }
    for (int q = 0; q < nq1; ++q) l1d[(size_t)2 * n1 * nq1 + q] = wg[q];
    for (int a = 0; a < 2 * n1; ++a) {
      l1d[(size_t)2 * n1 * nq1 + nq1 + a] = Le[a];
      l1d[(size_t)2 * n1 * nq1 + nq1 + 2 * n1 + a] = dLe[a];
    }
    if ((err = upload<double>(M, l1d, &M.t64.l1d)) != cudaSuccess) return DG_ERR_OOM;
    if ((err = upload<float>(M, l1d, &M.t32.l1d)) != cudaSuccess) return DG_ERR_OOM;
    int nt = 1;
    for (int k = 0; k < d; ++k) nt *= n1;
    std::vector<int> qi(nt, -1);
    for (size_t i = 0; i < modes.size(); ++i) {
      const auto& md = modes[i];   // md[k]: degree in direction k
      int t = 0;
      for (int k = d - 1; k >= 0; --k) t = t * n1 + md[k];   // t = a0 + n1 (a1 + n1 a2)
      qi[t] = (int)i;
    }
    if (cudaMalloc((void**)&M.qidx, sizeof(int) * nt) != cudaSuccess) return DG_ERR_OOM;
    M.allocs.push_back(M.qidx);
    if (cudaMemcpy(M.qidx, qi.data(), sizeof(int) * nt, cudaMemcpyHostToDevice) != cudaSuccess) return DG_ERR_CUDA;
  }
  if (cudaMalloc((void**)&M.status, sizeof(int)) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.status);
  if (cudaMemset(M.status, 0, sizeof(int)) != cudaSuccess) return DG_ERR_CUDA;
  if (cudaMalloc((void**)&M.scal, 16 * sizeof(double)) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.scal);
  if (cudaMalloc((void**)&M.partials, 2 * 1024 * sizeof(double)) != cudaSuccess) return DG_ERR_OOM;
  M.allocs.push_back(M.partials);
  if ((err = build_tc_tables(M)) != cudaSuccess)
    return err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  return DG_OK;
}

}  // namespace dgk

using namespace dgk;

extern "C" dg_status dg_mesh_create(const dg_mesh_desc* desc, const dg_physics* phys, void* stream,
                                    dg_mesh* out) {
  (void)stream;
  if (!out) return DG_ERR_INVALID;
  *out = nullptr;
  if (!desc || !phys) return DG_ERR_INVALID;
  if (desc->dim != 2 && desc->dim != 3) return DG_ERR_INVALID;
  if (desc->p < 0 || desc->p > 8) return DG_ERR_INVALID;
  if (desc->space != DG_SPACE_P && desc->space != DG_SPACE_Q) return DG_ERR_INVALID;
  int nq1 = desc->nq1d > 0 ? desc->nq1d : desc->p + 2;
  if (nq1 < desc->p + 1 || nq1 > 12) return DG_ERR_INVALID;
  long E = 1;
  for (int k = 0; k < desc->dim; ++k) {
    if (desc->n[k] < 1 || !(desc->hi[k] > desc->lo[k])) return DG_ERR_INVALID;
    E *= desc->n[k];
  }
  if (E > (1L << 26)) return DG_ERR_INVALID;
  if (!(phys->gamma > 1.0) || !(phys->Rgas > 0.0) || phys->mu < 0.0 || !(phys->Pr > 0.0) ||
      phys->roe_delta < 0.0 || phys->eta_br2 < 0.0)
    return DG_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  dg_mesh h = new dg_mesh_s();
  dg_status s = build_mesh(h->m, desc, phys);
  if (s == DG_OK) s = noalloc_prepare();
  if (s != DG_OK) {
    free_mesh(h->m);
    delete h;
    return s;
  }
  *out = h;
  return DG_OK;
}

extern "C" dg_status dg_mesh_destroy(dg_mesh mesh) {
  if (!mesh) return DG_ERR_INVALID;
  free_mesh(mesh->m);
  delete mesh;
  return DG_OK;
}

extern "C" dg_status dg_mesh_info(dg_mesh mesh, int* n_elem, int* n_modes, int* n_vars,
                                  size_t* n_dofs) {
  if (!mesh) return DG_ERR_INVALID;
  if (n_elem) *n_elem = mesh->m.E;
  if (n_modes) *n_modes = mesh->m.nm;
  if (n_vars) *n_vars = mesh->m.m;
  if (n_dofs) *n_dofs = (size_t)mesh->m.E * mesh->m.nb;
  return DG_OK;
}

extern "C" dg_status dg_status_sync(dg_mesh mesh, void* stream) {
  if (!mesh) return DG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  if (cudaMemcpyAsync(&h, mesh->m.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return DG_ERR_CUDA;
  if (cudaMemsetAsync(mesh->m.status, 0, sizeof(int), st) != cudaSuccess) return DG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DG_ERR_CUDA;
  if (h & ST_TIMEOUT) return DG_ERR_TIMEOUT;
  if (h & ST_NONPHYSICAL) return DG_ERR_NONPHYSICAL;
  if (h & (ST_SINGULAR | ST_NONFINITE)) return DG_ERR_BREAKDOWN;
  return DG_OK;
}
