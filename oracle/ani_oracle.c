/*
 * ani_oracle.c -- plain FP64 CPU oracle for the energy and forces of an
 * ANI-2x-style neural network potential (NNP).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it and shares no code, header, table or constant
 * with it.
 *
 * What it computes (the paper: Sec. 2 "Methods", Eqs. 2-3 -- the NNP term
 * V_NNP(Z, r) of the NNP region and its forces F = -grad V_NNP; Sec. 1 names
 * the model: the ANI modified Behler-Parrinello symmetry functions with the
 * 5.1 A cutoff, the elements H, C, N, O, F, S, Cl, and an 8-network ensemble
 * in Sec. 2 "Optimization").  The paper prints no equations for the
 * featurizer, so the functional form below is the ANI one, with the
 * hyper-parameters of the 24-atom single-molecule workload:
 *
 *   fc(r; Rc)  = 0.5 cos(pi r / Rc) + 0.5 for r < Rc, else 0
 *   radial     G_i[s, k]       = sum_{j: s(j)=s, r_ij<Rcr} 1/4 exp(-EtaR (r_ij - ShfR_k)^2) fc(r_ij; Rcr)
 *   angular    G_i[p(s,t), a, z] = sum_{j<k, r_ij<Rca, r_ik<Rca, {s(j),s(k)}={s,t}}
 *                 2 ((1 + cos(theta_ijk - ShfZ_z)) / 2)^Zeta
 *                 * exp(-EtaA ((r_ij + r_ik)/2 - ShfA_a)^2) fc(r_ij; Rca) fc(r_ik; Rca)
 *              with theta_ijk = acos(0.95 cos(angle j-i-k)).
 *   feature vector: [radial: species-major 7x16 | angular: 28 species-pair
 *              blocks (row-major upper triangle s<=t), each ShfA-major then ShfZ]
 *   network:   per element, h1 = celu(W1 G + b1), h2 = celu(W2 h1 + b2),
 *              h3 = celu(W3 h2 + b3), y = w4 . h3 + b4, celu alpha = 0.1
 *   energy:    E_mol = (1/M) sum_m sum_{i in mol} y_m(i)    (no self energies)
 *   forces:    F = -dE/dx by analytic reverse mode (below), checked against
 *              central finite differences by the test suite.
 *
 * Pair predicate: d^2 < Rc^2 in FP64 on the exact FP64 differences of the
 * input coordinates, with Rc the FP32 constant (5.1f, 3.5f) promoted to FP64
 * and every product/sum rounded separately (the file is built with
 * -ffp-contract=off).  Periodic boxes use the minimum image
 * d - L * floor(d / L + 0.5).
 *
 * Everything is FP64; weights arrive as FP32 and are promoted.
 *
 * Two models share the code through a model description (o_model): model 0
 * is the ANI-2x-shaped one above (7 elements, 1008 features); model 1 is the
 * ANI-1x-shaped one that the paper also runs (Sec. 3 "Extensibility with
 * other NNPs"): elements H, C, N, O; Rcr = 5.2 A, EtaR = 16, 16 radial shifts
 * 0.9 + 0.26875 k A; Rca = 3.5 A, EtaA = 8, Zeta = 32, 4 distance shifts
 * 0.9 + 0.65 a A and 8 angle shifts pi/16 + z pi/8 rad; 4x16 radial + 10
 * species-pair blocks of 4x8 = 384 features; networks H 384-160-128-96-1,
 * C 384-144-112-96-1, N and O 384-128-112-96-1 (the paper prints none of
 * these; they are the ANI-1x model's).
 *
 * The file also holds the NNP-MM coupling term of Eq. 4 (at its end), the
 * pair sum that couples the NNP region to the MM region.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_MAXSPEC 7
#define O_MAXSHF 16

static const double O_PI = 3.14159265358979323846;

/* A model: its elements, the featurizer's hyper-parameters and shift grids,
 * and the hidden widths of each element's network.  Feature layout:
 * [radial: species-major nspec x nshfr | angular: npairs species-pair blocks
 * (row-major upper triangle s <= t), each ShfA-major then ShfZ]. */
typedef struct {
  int nspec, nshfr, nshfa, nshfz;
  int nradial, npairs, nfeat;
  int z[O_MAXSPEC];
  int hidden[O_MAXSPEC][3];
  double Rcr, Rca, EtaR, EtaA, Zeta;
  double ShfR[O_MAXSHF], ShfA[O_MAXSHF], ShfZ[O_MAXSHF];
} o_model;

/* Model 0 (ANI-2x-shaped, shift grids as closed linspaces over the stated
 * ranges) or model 1 (ANI-1x-shaped); returns -1 for another id. */
static int o_model_init(o_model* M, int id) {
  int k, e;
  memset(M, 0, sizeof(*M));
  if (id == 0) {
    static const int z[7] = {1, 6, 7, 8, 9, 16, 17};
    static const int hid[7][3] = {{256, 192, 160}, {224, 192, 160}, {192, 160, 128}, {192, 160, 128},
                                  {160, 128, 96},  {160, 128, 96},  {160, 128, 96}};
    M->nspec = 7; M->nshfr = 16; M->nshfa = 8; M->nshfz = 4;
    for (e = 0; e < 7; ++e) { M->z[e] = z[e]; M->hidden[e][0] = hid[e][0]; M->hidden[e][1] = hid[e][1]; M->hidden[e][2] = hid[e][2]; }
    M->Rcr = (double)5.1f;  /* FP32 constant promoted (pair predicate) */
    M->Rca = (double)3.5f;
    M->EtaR = 19.7;
    M->EtaA = 12.5;
    M->Zeta = 14.1;
    for (k = 0; k < 16; ++k) M->ShfR[k] = 0.8 + (4.9 - 0.8) * k / 15;
    for (k = 0; k < 8; ++k) M->ShfA[k] = 0.8 + (3.1 - 0.8) * k / 7;
    for (k = 0; k < 4; ++k) M->ShfZ[k] = 0.39 + (2.75 - 0.39) * k / 3;
  } else if (id == 1) {
    static const int z[4] = {1, 6, 7, 8};
    static const int hid[4][3] = {{160, 128, 96}, {144, 112, 96}, {128, 112, 96}, {128, 112, 96}};
    M->nspec = 4; M->nshfr = 16; M->nshfa = 4; M->nshfz = 8;
    for (e = 0; e < 4; ++e) { M->z[e] = z[e]; M->hidden[e][0] = hid[e][0]; M->hidden[e][1] = hid[e][1]; M->hidden[e][2] = hid[e][2]; }
    M->Rcr = (double)5.2f;
    M->Rca = (double)3.5f;
    M->EtaR = 16.0;
    M->EtaA = 8.0;
    M->Zeta = 32.0;
    for (k = 0; k < 16; ++k) M->ShfR[k] = 0.9 + 0.26875 * k;
    for (k = 0; k < 4; ++k) M->ShfA[k] = 0.9 + 0.65 * k;
    for (k = 0; k < 8; ++k) M->ShfZ[k] = O_PI / 16.0 + k * O_PI / 8.0;
  } else {
    return -1;
  }
  M->nradial = M->nspec * M->nshfr;
  M->npairs = M->nspec * (M->nspec + 1) / 2;
  M->nfeat = M->nradial + M->npairs * M->nshfa * M->nshfz;
  return 0;
}

static int o_species(const o_model* M, int z) {
  int e;
  for (e = 0; e < M->nspec; ++e)
    if (M->z[e] == z) return e;
  return -1;
}

/* Index of the unordered species pair {s, t} (s <= t) in the row-major upper
 * triangle of an nspec x nspec matrix. */
static int o_pair_index(const o_model* M, int s, int t) {
  int a = s < t ? s : t, b = s < t ? t : s, idx = 0, r;
  for (r = 0; r < a; ++r) idx += M->nspec - r;
  return idx + (b - a);
}

/* Number of floats of one element's network: W1 b1 W2 b2 W3 b3 w4 b4. */
static long o_element_params(const o_model* M, int e) {
  const int n0 = M->nfeat, n1 = M->hidden[e][0], n2 = M->hidden[e][1], n3 = M->hidden[e][2];
  return (long)n1 * n0 + n1 + (long)n2 * n1 + n2 + (long)n3 * n2 + n3 + n3 + 1;
}

static long o_model_params(const o_model* M) {
  long s = 0;
  int e;
  for (e = 0; e < M->nspec; ++e) s += o_element_params(M, e);
  return s;
}

long ani_oracle_weights_per_model_m(int model) {
  o_model M;
  return o_model_init(&M, model) ? -1 : o_model_params(&M);
}
long ani_oracle_weights_per_model(void) { return ani_oracle_weights_per_model_m(0); }
int ani_oracle_num_features_m(int model) {
  o_model M;
  return o_model_init(&M, model) ? -1 : M.nfeat;
}
int ani_oracle_num_features(void) { return ani_oracle_num_features_m(0); }

/* Displacement x_j - x_i, minimum image when box != NULL. */
static void o_disp(const double* xi, const double* xj, const double* box, double out[3]) {
  int c;
  for (c = 0; c < 3; ++c) {
    double d = xj[c] - xi[c];
    if (box) {
      double L = box[c];
      double n = floor(d / L + 0.5);
      d = d - L * n;
    }
    out[c] = d;
  }
}

static double o_dist2(const double d[3]) {
  double s = d[0] * d[0];
  s = s + d[1] * d[1];
  s = s + d[2] * d[2];
  return s;
}

static double o_fc(double r, double rc) { return r < rc ? 0.5 * cos(O_PI * r / rc) + 0.5 : 0.0; }
static double o_dfc(double r, double rc) { return r < rc ? -0.5 * O_PI / rc * sin(O_PI * r / rc) : 0.0; }

static double o_celu(double x) {
  const double alpha = 0.1;
  double pos = x > 0.0 ? x : 0.0;
  double neg = alpha * (exp(x / alpha) - 1.0);
  return pos + (neg < 0.0 ? neg : 0.0);
}
static double o_dcelu(double x) { return x > 0.0 ? 1.0 : exp(x / 0.1); }

/* ------------------------------------------------------------------------ */
/* Pair and triple enumeration, brute force.                                 */

/* Ordered pairs (i, j), i != j, with d^2 < rc^2.  Returns the count (may
 * exceed cap; only the first cap are written). */
long ani_oracle_pairs(int n, const double* pos, const double* box, double rc,
                      int32_t* out_i, int32_t* out_j, long cap) {
  long cnt = 0;
  const double rc2 = rc * rc;
  int i, j;
  for (i = 0; i < n; ++i)
    for (j = 0; j < n; ++j) {
      double d[3];
      if (i == j) continue;
      o_disp(pos + 3 * i, pos + 3 * j, box, d);
      if (o_dist2(d) < rc2) {
        if (cnt < cap) { out_i[cnt] = i; out_j[cnt] = j; }
        ++cnt;
      }
    }
  return cnt;
}

/* Triples (i, j, k), j < k, j != i, k != i, both within rc of i. */
long ani_oracle_triples(int n, const double* pos, const double* box, double rc,
                        int32_t* out_i, int32_t* out_j, int32_t* out_k, long cap) {
  long cnt = 0;
  const double rc2 = rc * rc;
  int i, j, k;
  for (i = 0; i < n; ++i)
    for (j = 0; j < n; ++j) {
      double dj[3];
      if (j == i) continue;
      o_disp(pos + 3 * i, pos + 3 * j, box, dj);
      if (!(o_dist2(dj) < rc2)) continue;
      for (k = j + 1; k < n; ++k) {
        double dk[3];
        if (k == i) continue;
        o_disp(pos + 3 * i, pos + 3 * k, box, dk);
        if (!(o_dist2(dk) < rc2)) continue;
        if (cnt < cap) { out_i[cnt] = i; out_j[cnt] = j; out_k[cnt] = k; }
        ++cnt;
      }
    }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Featurizer of one molecule (atoms 0..n-1 of pos/spec).                    */

static void o_aev_molecule(const o_model* h, int n, const int* spec, const double* pos,
                           const double* box, double* aev /* [n][nfeat] */) {
  const double rcr2 = h->Rcr * h->Rcr, rca2 = h->Rca * h->Rca;
  int i, j, k, a, z, s;
  memset(aev, 0, sizeof(double) * (size_t)n * h->nfeat);
  for (i = 0; i < n; ++i) {
    double* G = aev + (size_t)i * h->nfeat;
    /* radial */
    for (j = 0; j < n; ++j) {
      double d[3], r, fc;
      if (j == i) continue;
      o_disp(pos + 3 * i, pos + 3 * j, box, d);
      if (!(o_dist2(d) < rcr2)) continue;
      r = sqrt(o_dist2(d));
      fc = o_fc(r, h->Rcr);
      for (s = 0; s < h->nshfr; ++s) {
        double x = r - h->ShfR[s];
        G[spec[j] * h->nshfr + s] += 0.25 * exp(-h->EtaR * x * x) * fc;
      }
    }
    /* angular */
    for (j = 0; j < n; ++j) {
      double dj[3], rj;
      if (j == i) continue;
      o_disp(pos + 3 * i, pos + 3 * j, box, dj);
      if (!(o_dist2(dj) < rca2)) continue;
      rj = sqrt(o_dist2(dj));
      for (k = j + 1; k < n; ++k) {
        double dk[3], rk, cos_t, theta, fcjk, u;
        double* blk;
        if (k == i) continue;
        o_disp(pos + 3 * i, pos + 3 * k, box, dk);
        if (!(o_dist2(dk) < rca2)) continue;
        rk = sqrt(o_dist2(dk));
        cos_t = (dj[0] * dk[0] + dj[1] * dk[1] + dj[2] * dk[2]) / (rj * rk);
        theta = acos(0.95 * cos_t);
        fcjk = o_fc(rj, h->Rca) * o_fc(rk, h->Rca);
        u = 0.5 * (rj + rk);
        blk = G + h->nradial + o_pair_index(h, spec[j], spec[k]) * (h->nshfa * h->nshfz);
        for (a = 0; a < h->nshfa; ++a) {
          double x = u - h->ShfA[a];
          double rad = exp(-h->EtaA * x * x);
          for (z = 0; z < h->nshfz; ++z) {
            double ang = 2.0 * pow(0.5 * (1.0 + cos(theta - h->ShfZ[z])), h->Zeta);
            blk[a * h->nshfz + z] += ang * rad * fcjk;
          }
        }
      }
    }
  }
}

/* Reverse mode of the featurizer: given g = dE/dG (per atom, nfeat each),
 * accumulate dE/dx into grad[n][3]. */
static void o_aev_adjoint(const o_model* h, int n, const int* spec, const double* pos,
                          const double* box, const double* g, double* grad) {
  const double rcr2 = h->Rcr * h->Rcr, rca2 = h->Rca * h->Rca;
  int i, j, k, a, z, s, c;
  for (i = 0; i < n; ++i) {
    const double* gi = g + (size_t)i * h->nfeat;
    /* radial: term = 1/4 exp(-EtaR (r - R)^2) fc(r) */
    for (j = 0; j < n; ++j) {
      double d[3], r, fc, dfc, dEdr = 0.0;
      if (j == i) continue;
      o_disp(pos + 3 * i, pos + 3 * j, box, d);
      if (!(o_dist2(d) < rcr2)) continue;
      r = sqrt(o_dist2(d));
      fc = o_fc(r, h->Rcr);
      dfc = o_dfc(r, h->Rcr);
      for (s = 0; s < h->nshfr; ++s) {
        double x = r - h->ShfR[s];
        double e = exp(-h->EtaR * x * x);
        double dterm = 0.25 * (e * (-2.0 * h->EtaR * x) * fc + e * dfc);
        dEdr += gi[spec[j] * h->nshfr + s] * dterm;
      }
      for (c = 0; c < 3; ++c) {
        grad[3 * j + c] += dEdr * d[c] / r;
        grad[3 * i + c] -= dEdr * d[c] / r;
      }
    }
    /* angular */
    for (j = 0; j < n; ++j) {
      double dj[3], rj;
      if (j == i) continue;
      o_disp(pos + 3 * i, pos + 3 * j, box, dj);
      if (!(o_dist2(dj) < rca2)) continue;
      rj = sqrt(o_dist2(dj));
      for (k = j + 1; k < n; ++k) {
        double dk[3], rk, cos_t, cp, theta, dtheta_dcp, fcj, fck, dfcj, dfck, u;
        double dE_dcos = 0.0, dE_drj = 0.0, dE_drk = 0.0;
        const double* gb;
        if (k == i) continue;
        o_disp(pos + 3 * i, pos + 3 * k, box, dk);
        if (!(o_dist2(dk) < rca2)) continue;
        rk = sqrt(o_dist2(dk));
        cos_t = (dj[0] * dk[0] + dj[1] * dk[1] + dj[2] * dk[2]) / (rj * rk);
        cp = 0.95 * cos_t;
        theta = acos(cp);
        dtheta_dcp = -1.0 / sqrt(1.0 - cp * cp);
        fcj = o_fc(rj, h->Rca);
        fck = o_fc(rk, h->Rca);
        dfcj = o_dfc(rj, h->Rca);
        dfck = o_dfc(rk, h->Rca);
        u = 0.5 * (rj + rk);
        gb = gi + h->nradial + o_pair_index(h, spec[j], spec[k]) * (h->nshfa * h->nshfz);
        for (a = 0; a < h->nshfa; ++a) {
          double x = u - h->ShfA[a];
          double rad = exp(-h->EtaA * x * x);
          double drad_du = rad * (-2.0 * h->EtaA * x);
          for (z = 0; z < h->nshfz; ++z) {
            double gv = gb[a * h->nshfz + z];
            double base = 0.5 * (1.0 + cos(theta - h->ShfZ[z]));
            double ang = 2.0 * pow(base, h->Zeta);
            /* d ang / d theta = 2 Zeta base^(Zeta-1) * (-sin(theta - ShfZ) / 2) */
            double dang_dtheta = -h->Zeta * pow(base, h->Zeta - 1.0) * sin(theta - h->ShfZ[z]);
            dE_dcos += gv * dang_dtheta * dtheta_dcp * 0.95 * rad * fcj * fck;
            dE_drj += gv * ang * (0.5 * drad_du * fcj * fck + rad * dfcj * fck);
            dE_drk += gv * ang * (0.5 * drad_du * fcj * fck + rad * fcj * dfck);
          }
        }
        /* d cos / d dj = dk/(rj rk) - cos dj / rj^2 ; d rj / d dj = dj / rj */
        for (c = 0; c < 3; ++c) {
          double gj = dE_dcos * (dk[c] / (rj * rk) - cos_t * dj[c] / (rj * rj)) + dE_drj * dj[c] / rj;
          double gk = dE_dcos * (dj[c] / (rj * rk) - cos_t * dk[c] / (rk * rk)) + dE_drk * dk[c] / rk;
          grad[3 * j + c] += gj;
          grad[3 * k + c] += gk;
          grad[3 * i + c] -= gj + gk;
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Atomic networks.                                                          */

/* One element network of one model: forward y(G) and, when dG != NULL,
 * accumulate scale * dy/dG into dG.  w points at this element's packed
 * parameters (W1 b1 W2 b2 W3 b3 w4 b4, W row-major [out][in]). */
static double o_network(const o_model* M, int e, const float* w, const double* G, double scale,
                        double* dG, double* work) {
  const int n0 = M->nfeat, n1 = M->hidden[e][0], n2 = M->hidden[e][1], n3 = M->hidden[e][2];
  const float *W1 = w, *b1 = W1 + (long)n1 * n0, *W2 = b1 + n1, *b2 = W2 + (long)n2 * n1,
              *W3 = b2 + n2, *b3 = W3 + (long)n3 * n2, *w4 = b3 + n3, *b4 = w4 + n3;
  double *z1 = work, *z2 = z1 + n1, *z3 = z2 + n2, *h1 = z3 + n3, *h2 = h1 + n1, *h3 = h2 + n2;
  double *d1 = h3 + n3, *d2 = d1 + n1, *d3 = d2 + n2;
  double y;
  int o, q;
  for (o = 0; o < n1; ++o) {
    double acc = b1[o];
    for (q = 0; q < n0; ++q) acc += (double)W1[(long)o * n0 + q] * G[q];
    z1[o] = acc;
    h1[o] = o_celu(acc);
  }
  for (o = 0; o < n2; ++o) {
    double acc = b2[o];
    for (q = 0; q < n1; ++q) acc += (double)W2[(long)o * n1 + q] * h1[q];
    z2[o] = acc;
    h2[o] = o_celu(acc);
  }
  for (o = 0; o < n3; ++o) {
    double acc = b3[o];
    for (q = 0; q < n2; ++q) acc += (double)W3[(long)o * n2 + q] * h2[q];
    z3[o] = acc;
    h3[o] = o_celu(acc);
  }
  y = b4[0];
  for (q = 0; q < n3; ++q) y += (double)w4[q] * h3[q];
  if (!dG) return y;
  /* reverse: dy/dh3 = w4 */
  for (o = 0; o < n3; ++o) d3[o] = scale * (double)w4[o] * o_dcelu(z3[o]);
  for (q = 0; q < n2; ++q) {
    double acc = 0.0;
    for (o = 0; o < n3; ++o) acc += (double)W3[(long)o * n2 + q] * d3[o];
    d2[q] = acc * o_dcelu(z2[q]);
  }
  for (q = 0; q < n1; ++q) {
    double acc = 0.0;
    for (o = 0; o < n2; ++o) acc += (double)W2[(long)o * n1 + q] * d2[o];
    d1[q] = acc * o_dcelu(z1[q]);
  }
  for (q = 0; q < n0; ++q) {
    double acc = 0.0;
    for (o = 0; o < n1; ++o) acc += (double)W1[(long)o * n0 + q] * d1[o];
    dG[q] += acc;
  }
  return y;
}

/* ------------------------------------------------------------------------ */
/* Whole batch.                                                              */

/*
 * Energies (and optionally forces, features, per-atom energies, dE/dG) of a
 * batch of molecules.  Molecule m owns atoms [mol_off[m], mol_off[m+1]).
 * pos: [N][3] FP64.  box: NULL or 3 edge lengths (orthorhombic, periodic).
 * weights: n_models * ani_oracle_weights_per_model() FP32 values, packed
 * [model][element H..Cl][W1 b1 W2 b2 W3 b3 w4 b4].
 * Returns 0, -1 for an unknown atomic number, -2 for bad sizes.
 */
int ani_oracle_compute_m(int model, int n_mols, const int32_t* mol_off, const int32_t* Z,
                         const double* pos, const double* box, int n_models, const float* weights,
                         long n_weights, double* E, double* F, double* aev_out, double* atomE_out,
                         double* dEdG_out, int nthreads) {
  o_model h;
  long per_model;
  long elem_off[O_MAXSPEC];
  int m, e, bad = 0, nf;
  long acc = 0;
  if (o_model_init(&h, model)) return -2;
  per_model = o_model_params(&h);
  nf = h.nfeat;
  if (n_mols < 0 || n_models < 1 || n_weights != per_model * n_models) return -2;
  for (e = 0; e < h.nspec; ++e) { elem_off[e] = acc; acc += o_element_params(&h, e); }
  for (m = 0; m < mol_off[n_mols]; ++m)
    if (o_species(&h, Z[m]) < 0) bad = 1;
  if (bad) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (m = 0; m < n_mols; ++m) {
    const int a0 = mol_off[m], n = mol_off[m + 1] - mol_off[m];
    int* spec = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    double* G = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nf);
    double* dG = (double*)calloc((size_t)(n > 0 ? n : 1) * nf, sizeof(double));
    double* grad = (double*)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
    double* work = (double*)malloc(sizeof(double) * 3 * (256 + 192 + 160));
    double Emol = 0.0;
    int i, mm, c;
    for (i = 0; i < n; ++i) spec[i] = o_species(&h, Z[a0 + i]);
    o_aev_molecule(&h, n, spec, pos + 3 * (size_t)a0, box, G);
    for (i = 0; i < n; ++i) {
      double ei = 0.0;
      for (mm = 0; mm < n_models; ++mm) {
        const float* w = weights + mm * per_model + elem_off[spec[i]];
        ei += o_network(&h, spec[i], w, G + (size_t)i * nf, 1.0 / n_models,
                        F ? dG + (size_t)i * nf : NULL, work);
      }
      ei /= n_models;
      if (atomE_out) atomE_out[a0 + i] = ei;
      Emol += ei;
    }
    E[m] = Emol;
    if (aev_out) memcpy(aev_out + (size_t)a0 * nf, G, sizeof(double) * (size_t)n * nf);
    if (dEdG_out && F) memcpy(dEdG_out + (size_t)a0 * nf, dG, sizeof(double) * (size_t)n * nf);
    if (F) {
      o_aev_adjoint(&h, n, spec, pos + 3 * (size_t)a0, box, dG, grad);
      for (i = 0; i < n; ++i)
        for (c = 0; c < 3; ++c) F[3 * (size_t)(a0 + i) + c] = -grad[3 * i + c];
    }
    free(spec); free(G); free(dG); free(grad); free(work);
  }
  return 0;
}

int ani_oracle_compute(int n_mols, const int32_t* mol_off, const int32_t* Z, const double* pos,
                       const double* box, int n_models, const float* weights, long n_weights,
                       double* E, double* F, double* aev_out, double* atomE_out,
                       double* dEdG_out, int nthreads) {
  return ani_oracle_compute_m(0, n_mols, mol_off, Z, pos, box, n_models, weights, n_weights, E, F,
                              aev_out, atomE_out, dEdG_out, nthreads);
}

/* Featurizer alone for one molecule (species given as atomic numbers). */
int ani_oracle_aev_m(int model, int n, const int32_t* Z, const double* pos, const double* box,
                     double* aev) {
  o_model h;
  int i;
  int* spec;
  if (o_model_init(&h, model)) return -2;
  spec = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (i = 0; i < n; ++i) {
    spec[i] = o_species(&h, Z[i]);
    if (spec[i] < 0) { free(spec); return -1; }
  }
  o_aev_molecule(&h, n, spec, pos, box, aev);
  free(spec);
  return 0;
}
int ani_oracle_aev(int n, const int32_t* Z, const double* pos, const double* box, double* aev) {
  return ani_oracle_aev_m(0, n, Z, pos, box, aev);
}

/* Featurizer adjoint alone: grad[n][3] += d(sum g . G)/dx for given g. */
int ani_oracle_aev_adjoint_m(int model, int n, const int32_t* Z, const double* pos,
                             const double* box, const double* g, double* grad) {
  o_model h;
  int i;
  int* spec;
  if (o_model_init(&h, model)) return -2;
  spec = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (i = 0; i < n; ++i) {
    spec[i] = o_species(&h, Z[i]);
    if (spec[i] < 0) { free(spec); return -1; }
  }
  o_aev_adjoint(&h, n, spec, pos, box, g, grad);
  free(spec);
  return 0;
}
int ani_oracle_aev_adjoint(int n, const int32_t* Z, const double* pos, const double* box,
                           const double* g, double* grad) {
  return ani_oracle_aev_adjoint_m(0, n, Z, pos, box, g, grad);
}

/* Hyper-parameters as the oracle uses them (for pins that check the grid):
 * Rcr Rca EtaR EtaA Zeta, then nshfr ShfR, nshfa ShfA, nshfz ShfZ. */
int ani_oracle_hyper_m(int model, double* out /* 5 + 3 x 16 */) {
  o_model h;
  int k;
  if (o_model_init(&h, model)) return -2;
  out[0] = h.Rcr; out[1] = h.Rca; out[2] = h.EtaR; out[3] = h.EtaA; out[4] = h.Zeta;
  for (k = 0; k < h.nshfr; ++k) out[5 + k] = h.ShfR[k];
  for (k = 0; k < h.nshfa; ++k) out[5 + h.nshfr + k] = h.ShfA[k];
  for (k = 0; k < h.nshfz; ++k) out[5 + h.nshfr + h.nshfa + k] = h.ShfZ[k];
  return 0;
}
void ani_oracle_hyper(double* out /* 5 + 16 + 8 + 4 */) { ani_oracle_hyper_m(0, out); }

/* ---------------------------------------------------------------------------
 * NNP-MM coupling term (Eq. 4, the mechanical-embedding scheme of Sec. 2):
 *
 *   V_NNP-MM = sum_{i in NNP} sum_{j in MM} ( V_C(i,j) + V_LJ(i,j) )
 *   V_C  = ke q_i q_j / r_ij                       (ke = 1 / (4 pi eps0) in the
 *                                                   caller's units)
 *   V_LJ = 4 eps_ij ((sigma_ij / r_ij)^12 - (sigma_ij / r_ij)^6)
 *   sigma_ij = (sigma_i + sigma_j) / 2,  eps_ij = sqrt(eps_i eps_j)
 *                                                  (Lorentz-Berthelot, the
 *                                                   rule of the GAFF2 / TIP3P
 *                                                   force fields of Sec. 3)
 *
 * every pair, no cutoff and no periodic images, as the equation is written.
 * Adds the energy to *energy and the forces -dV/dx to f_nnp [n_nnp][3] and
 * f_mm [n_mm][3].  For error bounds it can also add the sum of the squared
 * pair energies (e_sq) and, per atom, the sum of the magnitudes of its pair
 * forces (g_nnp, g_mm); null pointers skip them.  Returns -1 (and adds
 * nothing) if two atoms coincide.
 */
int ani_oracle_coupling(int n_nnp, const double* xn, const double* qn, const double* sn,
                        const double* en, int n_mm, const double* xm, const double* qm,
                        const double* sm, const double* em, double ke, double* energy,
                        double* f_nnp, double* f_mm, double* e_sq, double* g_nnp, double* g_mm) {
  int i, j, k;
  double e_sum = 0.0, e2_sum = 0.0;
  for (i = 0; i < n_nnp; ++i)
    for (j = 0; j < n_mm; ++j) {
      double d[3];
      for (k = 0; k < 3; ++k) d[k] = xm[3 * j + k] - xn[3 * i + k];
      if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] == 0.0) return -1;
    }
  for (i = 0; i < n_nnp; ++i) {
    for (j = 0; j < n_mm; ++j) {
      double d[3], r2, r, sig, eps, vc, sr, s6, s12, vlj, dvdr;
      for (k = 0; k < 3; ++k) d[k] = xm[3 * j + k] - xn[3 * i + k];  /* from i to j */
      r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      r = sqrt(r2);
      sig = 0.5 * (sn[i] + sm[j]);
      eps = sqrt(en[i] * em[j]);
      vc = ke * qn[i] * qm[j] / r;
      sr = sig / r;
      s6 = sr * sr * sr * sr * sr * sr;
      s12 = s6 * s6;
      vlj = 4.0 * eps * (s12 - s6);
      e_sum += vc + vlj;
      e2_sum += (vc + vlj) * (vc + vlj);
      /* dV/dr; d r / d x_j = d / r, d r / d x_i = -d / r */
      dvdr = -vc / r + 4.0 * eps * (-12.0 * s12 + 6.0 * s6) / r;
      for (k = 0; k < 3; ++k) {
        f_mm[3 * j + k] -= dvdr * d[k] / r;
        f_nnp[3 * i + k] += dvdr * d[k] / r;
      }
      if (g_nnp) g_nnp[i] += fabs(dvdr);
      if (g_mm) g_mm[j] += fabs(dvdr);
    }
  }
  *energy += e_sum;
  if (e_sq) *e_sq += e2_sum;
  return 0;
}
