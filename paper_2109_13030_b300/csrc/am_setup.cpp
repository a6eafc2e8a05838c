// Host-side FP64 setup of the batched AM loop: Bernstein basis, the constant
// KKT inverses of the position and heading QPs, and the constant block the
// kernels stage into shared memory.
//
// The position QP of one trajectory (Eq. zeta_1_sepration_1) splits into two
// identical 22-unknown problems, one per side: (c_x, c_c) and (c_y, c_s).
// Per side, F stacks [Pd 0; Pdd 0; (P, r_i P) for every circle i and obstacle
// j; 0 P] (display after Eq. ine_1), so F^T F has the closed block form
//   [Pd'Pd + Pdd'Pdd + n m P'P,   n (sum r_i) P'P      ]
//   [n (sum r_i) P'P,             (n sum r_i^2 + 1) P'P ]
// and the KKT matrix [Q + rho F'F, A'; A, 0] (Eq. over_2) is the same on both
// sides and for every trajectory: its inverse is formed once here, in FP64,
// and only its folded blocks reach the device (Eq. over_3).
#include <cmath>
#include <cstring>

#include "am_internal.h"

namespace trajam {

static double binomial(int n, int k)
{
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

static double ipow(double x, int e) { return e < 0 ? 0.0 : std::pow(x, e); }

// B_k(tau) = C(10,k) tau^k (1-tau)^(10-k), differentiated term by term with the
// product rule; d/dt = (1/T) d/dtau.
void bernstein_basis(int q, double T, std::vector<double> &P, std::vector<double> &Pd,
                     std::vector<double> &Pdd)
{
    const int N = NV - 1;
    P.assign(q * NV, 0.0);
    Pd.assign(q * NV, 0.0);
    Pdd.assign(q * NV, 0.0);
    for (int t = 0; t < q; ++t) {
        const double tau = q > 1 ? double(t) / double(q - 1) : 0.0, u = 1.0 - tau;
        for (int k = 0; k <= N; ++k) {
            const double c = binomial(N, k);
            const int a = k, b = N - k;
            double v = ipow(tau, a) * ipow(u, b);
            double d1 = 0.0, d2 = 0.0;
            if (a >= 1) d1 += a * ipow(tau, a - 1) * ipow(u, b);
            if (b >= 1) d1 -= b * ipow(tau, a) * ipow(u, b - 1);
            if (a >= 2) d2 += a * (a - 1) * ipow(tau, a - 2) * ipow(u, b);
            if (a >= 1 && b >= 1) d2 -= 2.0 * a * b * ipow(tau, a - 1) * ipow(u, b - 1);
            if (b >= 2) d2 += b * (b - 1) * ipow(tau, a) * ipow(u, b - 2);
            P[t * NV + k] = c * v;
            Pd[t * NV + k] = c * d1 / T;
            Pdd[t * NV + k] = c * d2 / (T * T);
        }
    }
}

// In-place Gauss-Jordan inverse with partial pivoting. Returns -1 if singular.
static int invert(std::vector<double> &A, int n)
{
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[p * n + j], A[c * n + j]);
                std::swap(I[p * n + j], I[c * n + j]);
            }
        const double inv = 1.0 / A[c * n + c];
        for (int j = 0; j < n; ++j) {
            A[c * n + j] *= inv;
            I[c * n + j] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[r * n + j] -= f * A[c * n + j];
                I[r * n + j] -= f * I[c * n + j];
            }
        }
    }
    A.swap(I);
    return 0;
}

static double inf_norm(const std::vector<double> &A, int n)
{
    double best = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += std::fabs(A[i * n + j]);
        best = std::max(best, s);
    }
    return best;
}

// cos(psi), sin(psi) and their first two time derivatives at both ends, from
// psi's boundary values by the chain rule.
static void slack_bc(const double psi_bc[6], double c_bc[6], double s_bc[6])
{
    for (int e = 0; e < 6; e += 3) {
        const double p = psi_bc[e], w = psi_bc[e + 1], al = psi_bc[e + 2];
        const double cp = std::cos(p), sp = std::sin(p);
        c_bc[e] = cp;
        s_bc[e] = sp;
        c_bc[e + 1] = -sp * w;
        s_bc[e + 1] = cp * w;
        c_bc[e + 2] = -cp * w * w - sp * al;
        s_bc[e + 2] = -sp * w * w + cp * al;
    }
}

// A: rows P[0], Pd[0], Pdd[0], P[q-1], Pd[q-1], Pdd[q-1] (Eq. reform_eq).
static void boundary_rows(const HostSetup &S, double A[6][NV])
{
    const int last = S.q - 1;
    for (int k = 0; k < NV; ++k) {
        A[0][k] = S.P[k];
        A[1][k] = S.Pd[k];
        A[2][k] = S.Pdd[k];
        A[3][k] = S.P[last * NV + k];
        A[4][k] = S.Pd[last * NV + k];
        A[5][k] = S.Pdd[last * NV + k];
    }
}

static std::vector<double> pos_kkt_inverse(const ProblemParams &pp, HostSetup &S, int &dim)
{
    double A[6][NV];
    boundary_rows(S, A);
    const int neq = pp.cs_boundary ? 12 : 6;
    dim = NS + neq;
    std::vector<double> K(dim * dim, 0.0);
    for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) {
            double v = pp.rho * S.FtF[a][b];
            if ((a < NV) == (b < NV)) v += S.H[a % NV][b % NV];
            K[a * dim + b] = v;
        }
    for (int blk = 0; blk < neq / 6; ++blk)
        for (int r = 0; r < 6; ++r)
            for (int k = 0; k < NV; ++k) {
                K[(NS + 6 * blk + r) * dim + blk * NV + k] = A[r][k];
                K[(blk * NV + k) * dim + NS + 6 * blk + r] = A[r][k];
            }
    const double nk = inf_norm(K, dim);
    if (invert(K, dim) != 0) return {};
    S.cond_pos = nk * inf_norm(K, dim);
    return K;
}

static std::vector<double> psi_kkt_inverse(const ProblemParams &pp, HostSetup &S)
{
    double A[6][NV];
    boundary_rows(S, A);
    const int dim = NV + 6;
    std::vector<double> K(dim * dim, 0.0);
    for (int a = 0; a < NV; ++a)
        for (int b = 0; b < NV; ++b) K[a * dim + b] = S.H[a][b] + pp.rho * S.PtP[a][b];
    for (int r = 0; r < 6; ++r)
        for (int k = 0; k < NV; ++k) {
            K[(NV + r) * dim + k] = A[r][k];
            K[k * dim + NV + r] = A[r][k];
        }
    const double nk = inf_norm(K, dim);
    if (invert(K, dim) != 0) return {};
    S.cond_psi = nk * inf_norm(K, dim);
    return K;
}

// Control points of a degree-10 Bernstein polynomial on [0, T] fixed by value,
// first and second derivative at both ends: x(0) = c_0, x'(0) = N (c_1 - c_0) / T,
// x''(0) = N (N-1) (c_2 - 2 c_1 + c_0) / T^2, and the mirror relations at t = T.
static void end_points(const double bc[6], double T, double out[6])
{
    const double N = NV - 1;
    out[0] = bc[0];
    out[1] = bc[0] + T * bc[1] / N;
    out[2] = 2.0 * out[1] - out[0] + T * T * bc[2] / (N * (N - 1));
    out[5] = bc[3];
    out[4] = bc[3] - T * bc[4] / N;
    out[3] = 2.0 * out[4] - out[5] + T * T * bc[5] / (N * (N - 1));
}

static void fold_boundary(const ProblemParams &pp, HostSetup &S, const std::vector<double> &Kp,
                          int dim, const std::vector<double> &Kq)
{
    double c_bc[6], s_bc[6];
    slack_bc(pp.psi_bc, c_bc, s_bc);
    end_points(pp.x_bc, pp.T, S.ends[0]);
    end_points(c_bc, pp.T, S.ends[1]);
    end_points(pp.y_bc, pp.T, S.ends[2]);
    end_points(s_bc, pp.T, S.ends[3]);
    end_points(pp.psi_bc, pp.T, S.ends[4]);
    const int neq = dim - NS;
    for (int side = 0; side < 2; ++side) {
        double b[12];
        const double *pos = side ? pp.y_bc : pp.x_bc;
        const double *sl = side ? s_bc : c_bc;
        for (int r = 0; r < 6; ++r) {
            b[r] = pos[r];
            b[6 + r] = sl[r];
        }
        for (int a = 0; a < NS; ++a) {
            double v = 0.0;
            for (int e = 0; e < neq; ++e) v += Kp[a * dim + NS + e] * b[e];
            S.kb[side][a] = v;
        }
    }
    const int dp = NV + 6;
    for (int a = 0; a < NV; ++a) {
        double v = 0.0;
        for (int e = 0; e < 6; ++e) v += Kq[a * dp + NV + e] * pp.psi_bc[e];
        S.kbpsi[a] = v;
    }
}

int build_setup(const ProblemParams &pp, int n, HostSetup &S)
{
    const int q = pp.q;
    S.q = q;
    S.n = n;
    bernstein_basis(q, pp.T, S.P, S.Pd, S.Pdd);
    double PdPd[NV][NV], PddPdd[NV][NV];
    for (int a = 0; a < NV; ++a)
        for (int b = 0; b < NV; ++b) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int t = 0; t < q; ++t) {
                s0 += S.P[t * NV + a] * S.P[t * NV + b];
                s1 += S.Pd[t * NV + a] * S.Pd[t * NV + b];
                s2 += S.Pdd[t * NV + a] * S.Pdd[t * NV + b];
            }
            S.PtP[a][b] = s0;
            PdPd[a][b] = s1;
            PddPdd[a][b] = s2;
            S.H[a][b] = s2;
        }
    double sr = 0.0, sr2 = 0.0;
    for (int i = 0; i < pp.m; ++i) {
        sr += pp.r[i];
        sr2 += pp.r[i] * pp.r[i];
    }
    for (int a = 0; a < NV; ++a)
        for (int b = 0; b < NV; ++b) {
            S.FtF[a][b] = PdPd[a][b] + PddPdd[a][b] + double(n) * pp.m * S.PtP[a][b];
            S.FtF[a][NV + b] = double(n) * sr * S.PtP[a][b];
            S.FtF[NV + a][b] = double(n) * sr * S.PtP[a][b];
            S.FtF[NV + a][NV + b] = (double(n) * sr2 + 1.0) * S.PtP[a][b];
        }
    int dim = 0;
    std::vector<double> Kp = pos_kkt_inverse(pp, S, dim);
    std::vector<double> Kq = psi_kkt_inverse(pp, S);
    if (Kp.empty() || Kq.empty()) return -1;
    for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) S.Minv[a][b] = Kp[a * dim + b];
    for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) {
            // Minv Q with Q = blockdiag(H, H): only the block of column b contributes
            const int blk = b / NV;
            double v = 0.0;
            for (int k = 0; k < NV; ++k) v += S.Minv[a][blk * NV + k] * S.H[k][b % NV];
            S.MQ[a][b] = v;
        }
    const int dp = NV + 6;
    for (int a = 0; a < NV; ++a)
        for (int b = 0; b < NV; ++b) S.Mpsi[a][b] = Kq[a * dp + b];
    for (int a = 0; a < NV; ++a)
        for (int b = 0; b < NV; ++b) {
            double v = 0.0;
            for (int k = 0; k < NV; ++k) v += S.Mpsi[a][k] * S.H[k][b];
            S.MpsiH[a][b] = v;
        }
    S.W.assign(q * NV, 0.0);
    for (int t = 0; t < q; ++t)
        for (int k = 0; k < NV; ++k) {
            double v = 0.0;
            for (int j = 0; j < NV; ++j) v += S.P[t * NV + j] * S.Mpsi[k][j];
            S.W[t * NV + k] = v;
        }
    fold_boundary(pp, S, Kp, dim, Kq);
    S.Kp.swap(Kp);
    S.Kq.swap(Kq);
    S.kdim = dim;
    return 0;
}

int rebuild_boundary(const ProblemParams &pp, HostSetup &S)
{
    // The KKT matrices depend on the basis, rho, n and the boundary rows A,
    // not on b: re-fold with the inverses formed by build_setup.
    if (S.Kp.empty() || S.Kq.empty()) return -1;
    fold_boundary(pp, S, S.Kp, S.kdim, S.Kq);
    return 0;
}

void bernstein_eval(const float *c, double T, double t, double out[3])
{
    const int n = NV - 1;
    double tau = t / T;
    tau = tau < 0 ? 0 : tau > 1 ? 1 : tau;
    auto basis = [&](int k, int deg) { return binomial(deg, k) * ipow(tau, k) * ipow(1 - tau, deg - k); };
    double v = 0, d = 0, dd = 0;
    for (int k = 0; k <= n; ++k) v += double(c[k]) * basis(k, n);
    // derivatives through the first and second differences of the control points
    for (int k = 0; k < n; ++k) d += (double(c[k + 1]) - c[k]) * basis(k, n - 1);
    for (int k = 0; k < n - 1; ++k) dd += (double(c[k + 2]) - 2.0 * c[k + 1] + c[k]) * basis(k, n - 2);
    out[0] = v;
    out[1] = d * n / T;
    out[2] = dd * n * (n - 1) / (T * T);
}

void init_cov_factor(double Lc[25])
{
    // R = D2^T D2 on the 11 control points, restricted to points 3..7
    double R[NV][NV] = {};
    for (int k = 0; k + 2 < NV; ++k) {
        const double w[3] = {1.0, -2.0, 1.0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) R[k + a][k + b] += w[a] * w[b];
    }
    std::vector<double> C(25);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) C[i * 5 + j] = R[3 + i][3 + j];
    invert(C, 5);  // R restricted to 3..7 is positive definite
    double dmax = 0;
    for (int i = 0; i < 5; ++i) dmax = std::fmax(dmax, C[i * 5 + i]);
    for (double &v : C) v /= dmax;
    // Cholesky C = L L^T
    for (int i = 0; i < 25; ++i) Lc[i] = 0.0;
    for (int j = 0; j < 5; ++j) {
        double s = C[j * 5 + j];
        for (int k = 0; k < j; ++k) s -= Lc[j * 5 + k] * Lc[j * 5 + k];
        Lc[j * 5 + j] = std::sqrt(s);
        for (int i = j + 1; i < 5; ++i) {
            double t = C[i * 5 + j];
            for (int k = 0; k < j; ++k) t -= Lc[i * 5 + k] * Lc[j * 5 + k];
            Lc[i * 5 + j] = t / Lc[j * 5 + j];
        }
    }
}

void shift_matrix(double s, double S[121])
{
    // column j: the new control points of the polynomial whose old control
    // points are the unit vector e_j; new point k is the blossom at
    // (s x (10 - k), (1 + s) x k), one de Casteljau level per argument
    for (int j = 0; j < NV; ++j)
        for (int k = 0; k < NV; ++k) {
            double c[NV];
            for (int i = 0; i < NV; ++i) c[i] = i == j ? 1.0 : 0.0;
            for (int lev = 0; lev < NV - 1; ++lev) {
                const double u = lev < NV - 1 - k ? s : 1.0 + s;
                for (int i = 0; i < NV - 1 - lev; ++i) c[i] = (1.0 - u) * c[i] + u * c[i + 1];
            }
            S[k * NV + j] = c[0];
        }
}

static int align4(int x) { return (x + 3) & ~3; }

ConstLayout make_layout(int q, int m, int n)
{
    ConstLayout L;
    std::memset(&L, 0, sizeof(L));
    L.q = q;
    L.m = m;
    L.n = n;
    // Per-step columns are zero-padded to a multiple of 8 steps (the k-step of
    // the tensor-core contractions), and the stride is 4 mod 8 so that eight
    // rows read at the same column offset, and 128-bit loads of consecutive
    // columns, fall on distinct banks.
    const int qs = ((q + 7) & ~7) + 4;
    L.qs = qs;
    int o = 0;
    // FP32 columns for the plain loop, outside the part the fused kernel stages
    L.off_pcol = o; o = align4(o + 3 * NV * qs);
    L.off_wcol = o; o = align4(o + NV * qs);
    // Split (hi, lo) columns: a stride of qp pairs = 16 mod 32 words, so the
    // 128-bit fragment loads of two neighbouring rows fall on distinct banks.
    int qp = (q + 7) & ~7;
    if (qp % 16 == 0) qp += 8;
    L.qp = qp;
    L.off_fused = o;
    L.off_prow = o; o = align4(o + 3 * q * 12);
    L.off_pcol2 = o; o = align4(o + 3 * NV * 2 * qp);
    L.off_mt = o; o = align4(o + NS * 24);
    L.off_mq = o; o = align4(o + NS * 24);
    L.off_ends = o; o = align4(o + 5 * 8);
    L.off_kb = o; o = align4(o + 2 * 24);
    L.off_mpsi = o; o = align4(o + NV * 12);
    L.off_mpsih = o; o = align4(o + NV * 12);
    L.off_ptp = o; o = align4(o + NV * 12);
    L.off_kbpsi = o; o = align4(o + 12);
    L.off_obs = o; o = align4(o + n * 2 * qs);
    L.off_obc = o; o = align4(o + n * 4);
    L.off_obt = o; o = align4(o + n);
    L.off_obs2 = o; o = align4(o + n * 2 * qs);
    L.off_obc2 = o; o = align4(o + n * 8);
    L.total = o;
    return L;
}

namespace {

// x = hi + lo with hi, lo both TF32 (round to nearest on the bit pattern:
// add half a TF32 unit to the magnitude bits, clear the 13 low mantissa
// bits), stored as FP32 values.  The fused kernel splits its run-time
// operands the same way.
void split_tf32(float x, float &hi, float &lo)
{
    auto round = [](float v) {
        uint32_t b;
        std::memcpy(&b, &v, 4);
        b = (b + 0x1000u) & 0xFFFFE000u;
        float r;
        std::memcpy(&r, &b, 4);
        return r;
    };
    hi = round(x);
    lo = round(x - hi);
}

void put_split(std::vector<float> &blob, int off, float v)
{
    split_tf32(v, blob[off], blob[off + 1]);
}

}  // namespace

void fill_constants(const HostSetup &S, const ProblemParams &pp, const ConstLayout &L,
                    std::vector<float> &blob)
{
    blob.assign(L.total, 0.0f);
    const int q = L.q, qs = L.qs;
    const std::vector<double> *B3[3] = {&S.P, &S.Pd, &S.Pdd};
    for (int b = 0; b < 3; ++b)
        for (int t = 0; t < q; ++t)
            for (int k = 0; k < NV; ++k) {
                const float v = float((*B3[b])[t * NV + k]);
                blob[L.off_prow + (b * q + t) * 12 + k] = v;
                blob[L.off_pcol + (b * NV + k) * qs + t] = v;
                put_split(blob, L.off_pcol2 + 2 * ((b * NV + k) * L.qp + t), v);
            }
    for (int t = 0; t < q; ++t)
        for (int k = 0; k < NV; ++k) {
            const float w = float(S.W[t * NV + k]);
            blob[L.off_wcol + k * qs + t] = w;
        }
    for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) {
            blob[L.off_mt + b * 24 + a] = float(S.Minv[a][b]);
            blob[L.off_mq + b * 24 + a] = float(S.MQ[a][b]);
        }
    for (int blk = 0; blk < 5; ++blk)
        for (int e = 0; e < 6; ++e) blob[L.off_ends + blk * 8 + e] = float(S.ends[blk][e]);
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < NS; ++a) blob[L.off_kb + s * 24 + a] = float(S.kb[s][a]);
    for (int a = 0; a < NV; ++a) {
        for (int b = 0; b < NV; ++b) {
            blob[L.off_mpsi + b * 12 + a] = float(S.Mpsi[a][b]);
            blob[L.off_mpsih + b * 12 + a] = float(S.MpsiH[a][b]);
            blob[L.off_ptp + b * 12 + a] = float(S.PtP[a][b]);
        }
        blob[L.off_kbpsi + a] = float(S.kbpsi[a]);
    }
}

}  // namespace trajam
