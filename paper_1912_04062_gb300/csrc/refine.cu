// refine.cu -- FP64 eigenpair refinement of the mixed form (not in the paper).
//
// Iterative refinement of Ogita and Aishima ("Iterative refinement for
// symmetric eigenvalue decomposition", 2018) applied to the Hermitian
// H = -iA (H z = lambda z  <=>  A z = i lambda z) with the full basis
// Zh = [Z, conj(Z)] (eigenvalues lambda and -lambda; n even, nev = n/2), in
// real arithmetic on M = [X Y] (Z = X + iY):
//   R = I - Zh^H Zh,  S = Zh^H H Zh,
//   lambda~_i = S_ii / (1 - R_ii),
//   E_ij = (S_ij + lambda~_j R_ij) / (lambda~_j - lambda~_i)  for separated pairs,
//   E_ij = R_ij / 2                                         otherwise,
//   Zh <- Zh + Zh E.
// Only Z's half is formed: Z <- Z + Z E11 + conj(Z) E21.  With
// Wg = M^T M and T = M^T A M (both n x n, computed to FP64 accuracy by the
// digit-slice tensor-core product), the blocks are
//   G  = Z^H Z = (XX + YY) + i (XY - YX),   F  = Z^T Z = (XX - YY) + i (XY + YX),
//   Sg = Z^H H Z = (T_XY - T_YX) - i (T_XX + T_YY),
//   Sf = Z^T H Z = (T_XY + T_YX) + i (T_YY - T_XX),
//   R11 = I - G, R21 = -F, E11 from (Sg, R11), E21 from (Sf, R21) with
//   denominators lambda~_j - lambda~_i and lambda~_j + lambda~_i,
// and the update is one real product M <- M + M U,
//   U = [[Er + Fr, Ei + Fi], [Fi - Ei, Er - Fr]]   (E11 = Er + i Ei, E21 = Fr + i Fi).
// A pair counts as separated when the first-order rotation it asks for is
// small: |lambda~_j - lambda~_i| > max(tau, rho (|S_ij| + |lambda~_j| |R_ij|)).
// Runs of neighbours that are not separated for the cluster factor rho (1024
// by default) form clusters; each cluster gets
// a Rayleigh-Ritz rotation from its FP64-accurate Gram and projection blocks
// (after Ogita and Aishima's treatment of clustered eigenvalues, 2019), and
// the first-order terms coupling it to other columns rotate with it.
#include <cfloat>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

// Full skew S (n x n, column-major) from the strict lower triangle of A:
// tiles below the diagonal are copied, tiles above are the negated transpose
// of their mirror (read coalesced through shared memory).
__global__ void skew_full_kernel(int n, const double* __restrict__ A, int lda, double* __restrict__ S) {
    __shared__ double tile[32][33];
    const int bi = blockIdx.x, bj = blockIdx.y;
    const int i0 = bi * 32, j0 = bj * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (bi >= bj) {
        for (int jj = ty; jj < 32; jj += 8) {
            const int i = i0 + tx, j = j0 + jj;
            if (i < n && j < n)
                S[(long long)j * n + i] = (i > j) ? A[(long long)j * lda + i]
                                                  : (i == j ? 0.0 : -A[(long long)i * lda + j]);
        }
    } else {
        for (int ii = ty; ii < 32; ii += 8) {
            const int j = j0 + tx, i = i0 + ii;  // A(j, i), j > i
            tile[ii][tx] = (i < n && j < n) ? A[(long long)i * lda + j] : 0.0;
        }
        __syncthreads();
        for (int jj = ty; jj < 32; jj += 8) {
            const int i = i0 + tx, j = j0 + jj;
            if (i < n && j < n) S[(long long)j * n + i] = -tile[tx][jj];
        }
    }
}

struct RefineScalars {
    unsigned long long emax_bits;  // max |E| over off-diagonal separated pairs (as double bits)
    unsigned int nclose;           // pairs neither separated nor inside one cluster
    double lmax;
    double rnorm2;                 // sum |R~_ij|^2 over the E11 block (orthogonality before the update)
    unsigned long long where;      // packed location of the max: i | j << 20 | blk << 40
    unsigned long long umax_bits;  // max |U_ij| of the update (as double bits)
    // the iteration's control on the device (no host round trip): once done is
    // set the remaining launches of the loop return at once
    int done;
    int su;            // digit slices of this iteration's update product
    RefineInfo hist;   // per-iteration record, copied to the host at the end
};

SK_DEV double refine_tau(int n, const RefineScalars* sc) { return 64.0 * n * DBL_EPSILON * sc->lmax; }

constexpr int KC = 16;  // largest cluster handled by Rayleigh-Ritz

struct cplx {
    double r, i;
};
SK_DEV cplx cmul(cplx a, cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
SK_DEV cplx cconj(cplx a) { return {a.r, -a.i}; }
SK_DEV cplx cadd(cplx a, cplx b) { return {a.r + b.r, a.i + b.i}; }
SK_DEV cplx csub(cplx a, cplx b) { return {a.r - b.r, a.i - b.i}; }
SK_DEV cplx cscale(cplx a, double s) { return {a.r * s, a.i * s}; }

// Blocks of Zh^H Zh and Zh^H H Zh at (i, j) (see the header comment).  Wg
// and T are formed on their lower triangle only and read as exactly symmetric
// and exactly skew: the correction's orthogonality identity
// E_ij + conj(E_ji) = R_ij holds only for an exactly Hermitian S and G.
struct Blocks {
    cplx G, F, Sg, Sf;
};
SK_DEV double wsym(const double* __restrict__ Wg, long long ld, int a, int b) {
    return a >= b ? Wg[a + b * ld] : Wg[b + a * ld];
}
SK_DEV double tskew(const double* __restrict__ T, long long ld, int a, int b) {
    return a > b ? T[a + b * ld] : (a < b ? -T[b + a * ld] : 0.0);
}
// lambda~_i = Sg_ii / G_ii = (T_XY - T_YX)_ii / (XX + YY)_ii
__global__ void refine_lambda_kernel(int m, int n, const double* __restrict__ Wg, const double* __restrict__ T,
                                     double* __restrict__ lt, const int* __restrict__ skip) {
    if (*skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long ld = n;
    const double g = Wg[i + i * ld] + Wg[(m + i) + (m + i) * ld];
    const double s = 2.0 * tskew(T, ld, i, m + i);  // (T_XY - T_YX)(i, i)
    lt[i] = s / g;
}

SK_DEV Blocks blocks(int i, int j, int m, long long ld, const double* __restrict__ Wg, const double* __restrict__ T) {
    const double XX = wsym(Wg, ld, i, j), YY = wsym(Wg, ld, m + i, m + j);
    const double XY = wsym(Wg, ld, i, m + j), YX = wsym(Wg, ld, m + i, j);
    const double TXX = tskew(T, ld, i, j), TYY = tskew(T, ld, m + i, m + j);
    const double TXY = tskew(T, ld, i, m + j), TYX = tskew(T, ld, m + i, j);
    Blocks b;
    b.G = {XX + YY, XY - YX};
    b.F = {XX - YY, XY + YX};
    b.Sg = {TXY - TYX, -(TXX + TYY)};
    b.Sf = {TXY + TYX, TYY - TXX};
    return b;
}

// first-order rotation the pair (i, j) asks for is small enough for the
// correction formula: |l_j - l_i| > max(tau, rho (|Sg_ij| + |l_j| |R_ij|)).
// Neighbours closer than that for the cluster factor rho form Rayleigh-Ritz
// clusters; every other pair takes the first-order formula when it asks for a
// rotation below 1/RHO1 (else E_ij = R_ij / 2, left to the next iteration).
constexpr double RHO1 = 64.0;
SK_DEV bool separated(double li, double lj, cplx Sg, cplx R, double tau, double rho) {
    const double need = rho * (hypot(Sg.r, Sg.i) + fabs(lj) * hypot(R.r, R.i));
    return fabs(lj - li) > fmax(tau, need);
}

// close[i] = 1 when the neighbours i and i+1 (eigenvalues sorted descending)
// are not separated
__global__ void refine_close_kernel(int m, int n, const double* __restrict__ Wg, const double* __restrict__ T,
                                    const double* __restrict__ lt, const RefineScalars* sc, double rho,
                                    int* __restrict__ close) {
    if (sc->done) return;
    const double tau = refine_tau(n, sc);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int c = 0;
    if (i + 1 < m) {
        const Blocks b = blocks(i, i + 1, m, n, Wg, T);
        const cplx R = {-b.G.r, -b.G.i};
        c = !separated(lt[i], lt[i + 1], b.Sg, R, tau, rho);
    }
    close[i] = c;
}

// One block (one working thread, shared-memory scratch) per index c0; c0 acts
// when it starts a cluster (a maximal run of close neighbours, 2 <= k <= KC):
// Rayleigh-Ritz on span(z_c0..z_c1-1) with the FP64-accurate Gram G_C and
// projection S_C: Cholesky G_C = L L^H, K = L^-1 S_C L^-H, cyclic complex
// Jacobi K = W diag(mu) W^H, V_C = L^-H W.  The cluster's columns become
// Z_C V_C; V_C (k x k, complex) is stored row-major per member in Vc, the
// Ritz values (descending) replace lt, and cid marks the members.
__global__ void refine_rr_kernel(int m, int n, const double* __restrict__ Wg, const double* __restrict__ T,
                                 const int* __restrict__ close, double* __restrict__ lt, int* __restrict__ cid,
                                 double* __restrict__ Vc, int* __restrict__ nbig, const int* __restrict__ skip) {
    __shared__ cplx L[KC][KC], K[KC][KC], W[KC][KC];
    if (*skip) return;
    const int c0 = blockIdx.x;
    if (c0 >= m || threadIdx.x != 0) return;
    const bool start = close[c0] && (c0 == 0 || !close[c0 - 1]);
    if (!start) {
        if (!close[c0] && (c0 == 0 || !close[c0 - 1])) cid[c0] = -1;
        return;
    }
    int c1 = c0 + 1;
    while (c1 < m && close[c1 - 1]) c1++;
    const int k = c1 - c0;
    if (k > KC) {
        for (int q = c0; q < c1; q++) cid[q] = -1;
        atomicAdd(nbig, 1);
        return;
    }
    // Gram and projection of the cluster
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) {
            const Blocks bl = blocks(c0 + a, c0 + b, m, n, Wg, T);
            L[a][b] = bl.G;
            K[a][b] = bl.Sg;
        }
    // Cholesky G = L L^H (lower)
    for (int j = 0; j < k; j++) {
        double d = L[j][j].r;
        for (int p = 0; p < j; p++) d -= L[j][p].r * L[j][p].r + L[j][p].i * L[j][p].i;
        d = sqrt(fmax(d, 1e-300));
        L[j][j] = {d, 0.0};
        for (int i = j + 1; i < k; i++) {
            cplx s = L[i][j];
            for (int p = 0; p < j; p++) s = csub(s, cmul(L[i][p], cconj(L[j][p])));
            L[i][j] = cscale(s, 1.0 / d);
        }
        for (int i = 0; i < j; i++) L[i][j] = {0.0, 0.0};
    }
    // K <- L^-1 K L^-H (forward substitution on columns, then on rows)
    for (int b = 0; b < k; b++)
        for (int i = 0; i < k; i++) {
            cplx s = K[i][b];
            for (int p = 0; p < i; p++) s = csub(s, cmul(L[i][p], K[p][b]));
            K[i][b] = cscale(s, 1.0 / L[i][i].r);
        }
    for (int a = 0; a < k; a++)
        for (int j = 0; j < k; j++) {
            cplx s = K[a][j];
            for (int p = 0; p < j; p++) s = csub(s, cmul(K[a][p], cconj(L[j][p])));
            K[a][j] = cscale(s, 1.0 / L[j][j].r);
        }
    // symmetrise (Hermitian up to rounding)
    for (int a = 0; a < k; a++) {
        K[a][a].i = 0.0;
        for (int b = a + 1; b < k; b++) {
            const cplx h = cscale(cadd(K[a][b], cconj(K[b][a])), 0.5);
            K[a][b] = h;
            K[b][a] = cconj(h);
        }
    }
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) W[a][b] = {a == b ? 1.0 : 0.0, 0.0};
    // cyclic Jacobi for the Hermitian K
    for (int sweep = 0; sweep < 30; sweep++) {
        double off = 0.0, dia = 0.0;
        for (int a = 0; a < k; a++) {
            dia += K[a][a].r * K[a][a].r;
            for (int b = a + 1; b < k; b++) off += K[a][b].r * K[a][b].r + K[a][b].i * K[a][b].i;
        }
        if (off <= 1e-34 * dia || off == 0.0) break;
        for (int p = 0; p < k - 1; p++)
            for (int q = p + 1; q < k; q++) {
                const double apq = hypot(K[p][q].r, K[p][q].i);
                if (apq == 0.0) continue;
                const cplx ph = cscale(K[p][q], 1.0 / apq);  // K_pq = apq e^{i phi}
                const double theta = 0.5 * atan2(2.0 * apq, K[q][q].r - K[p][p].r);
                const double c = cos(theta), s = sin(theta);
                // rotation J: columns p, q -> c e_p - s conj(ph)... (unitary, zeroes K_pq)
                const cplx sp = cscale(ph, s);  // s e^{i phi}
                for (int r = 0; r < k; r++) {   // K <- K J
                    const cplx kp = K[r][p], kq = K[r][q];
                    K[r][p] = csub(cscale(kp, c), cmul(kq, cconj(sp)));
                    K[r][q] = cadd(cmul(kp, sp), cscale(kq, c));
                    const cplx wp = W[r][p], wq = W[r][q];
                    W[r][p] = csub(cscale(wp, c), cmul(wq, cconj(sp)));
                    W[r][q] = cadd(cmul(wp, sp), cscale(wq, c));
                }
                for (int r = 0; r < k; r++) {   // K <- J^H K
                    const cplx kp = K[p][r], kq = K[q][r];
                    K[p][r] = csub(cscale(kp, c), cmul(sp, kq));
                    K[q][r] = cadd(cmul(cconj(sp), kp), cscale(kq, c));
                }
                K[p][q] = {0.0, 0.0};
                K[q][p] = {0.0, 0.0};
                K[p][p].i = 0.0;
                K[q][q].i = 0.0;
            }
    }
    // order Ritz values descending
    int ord[KC];
    for (int a = 0; a < k; a++) ord[a] = a;
    for (int a = 1; a < k; a++) {
        int t = ord[a], b = a - 1;
        while (b >= 0 && K[ord[b]][ord[b]].r < K[t][t].r) { ord[b + 1] = ord[b]; b--; }
        ord[b + 1] = t;
    }
    // V = L^-H W (back substitution with L^H), columns in Ritz order
    for (int col = 0; col < k; col++) {
        const int w = ord[col];
        cplx x[KC];
        for (int i = k - 1; i >= 0; i--) {
            cplx s = W[i][w];
            for (int p = i + 1; p < k; p++) s = csub(s, cmul(cconj(L[p][i]), x[p]));
            x[i] = cscale(s, 1.0 / L[i][i].r);
        }
        for (int i = 0; i < k; i++) {
            Vc[((long long)(c0 + i) * KC + col) * 2 + 0] = x[i].r;
            Vc[((long long)(c0 + i) * KC + col) * 2 + 1] = x[i].i;
        }
        lt[c0 + col] = K[w][w].r;
    }
    for (int q = c0; q < c1; q++) cid[q] = c0;
}

// Rotation B (block diagonal: V_C on each Rayleigh-Ritz cluster, 1 elsewhere):
// member list of index i and the entries B[a][i].
SK_DEV int basis_of(int i, int m, const int* __restrict__ cid, const double* __restrict__ Vc, int* idx, cplx* coef) {
    const int c = cid[i];
    if (c < 0) {
        idx[0] = i;
        coef[0] = {1.0, 0.0};
        return 1;
    }
    int k = 0;
    for (int a = c; a < m && cid[a] == c && k < KC; a++, k++) {
        idx[k] = a;
        coef[k] = {Vc[((long long)a * KC + (i - c)) * 2], Vc[((long long)a * KC + (i - c)) * 2 + 1]};
    }
    return k;
}

// First-order corrections in the rotated basis Z B:
//   Sg~ = B^H Sg B, G~ = B^H G B, Sf~ = B^T Sf B, F~ = B^T F B,
//   E~11 = OA(Sg~, I - G~) with denominators l_j - l_i,
//   E~21 = OA(Sf~, -F~) with denominators l_j + l_i,
// l = Ritz values on clusters, Rayleigh quotients elsewhere.  Stored as four
// m x m planes of Et (E~11 real, imag, E~21 real, imag).
__global__ void refine_etilde_kernel(int m, int n, const double* __restrict__ Wg, const double* __restrict__ T,
                                     const double* __restrict__ lt, const int* __restrict__ cid,
                                     const double* __restrict__ Vc, double* __restrict__ Et,
                                     RefineScalars* sc) {
    if (sc->done) return;
    const double tau = refine_tau(n, sc);
    const long long ld = n, mm = (long long)m * m;
    // largest |E|^2 (the square root is taken once, after the loop)
    double emax2 = 0.0, rn2 = 0.0;
    unsigned int close = 0;
    unsigned long long wloc = 0;
    // element (i, j), e = j m + i: threads along i, the grid's y along j (no
    // 64-bit division per element)
    for (int j = blockIdx.y; j < m; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const long long e = (long long)j * m + i;
        const double li = lt[i], lj = lt[j];
        cplx Sg, G, Sf, F;
        if (cid[i] < 0 && cid[j] < 0) {
            // neither index belongs to a cluster: B is the identity there, and
            // the rotated blocks are the blocks themselves
            const Blocks bl = blocks(i, j, m, ld, Wg, T);
            Sg = bl.Sg;
            G = bl.G;
            Sf = bl.Sf;
            F = bl.F;
        } else {
            int ia[KC], ja[KC];
            cplx ic[KC], jc[KC];
            const int ki = basis_of(i, m, cid, Vc, ia, ic);
            const int kj = basis_of(j, m, cid, Vc, ja, jc);
            Sg = G = Sf = F = cplx{0, 0};
            for (int a = 0; a < ki; a++)
                for (int b = 0; b < kj; b++) {
                    const Blocks bl = blocks(ia[a], ja[b], m, ld, Wg, T);
                    const cplx h = cmul(cconj(ic[a]), jc[b]);   // conj(B_ai) B_bj
                    const cplx t = cmul(ic[a], jc[b]);          // B_ai B_bj
                    Sg = cadd(Sg, cmul(h, bl.Sg));
                    G = cadd(G, cmul(h, bl.G));
                    Sf = cadd(Sf, cmul(t, bl.Sf));
                    F = cadd(F, cmul(t, bl.F));
                }
        }
        const bool same = (cid[i] >= 0 && cid[i] == cid[j]);
        const cplx R = {(i == j ? 1.0 : 0.0) - G.r, -G.i};
        cplx E11, E21;
        rn2 += R.r * R.r + R.i * R.i;
        if (i != j && !same && separated(li, lj, Sg, R, tau, RHO1)) {
            const double d = lj - li;
            E11 = {(Sg.r + lj * R.r) / d, (Sg.i + lj * R.i) / d};
            const double a = E11.r * E11.r + E11.i * E11.i;
            if (a > emax2) { emax2 = a; wloc = (unsigned long long)i | ((unsigned long long)j << 20); }
        } else {
            E11 = cscale(R, 0.5);
            if (i != j && !same) close++;
        }
        const cplx num = {Sf.r - lj * F.r, Sf.i - lj * F.i};
        const double d2 = lj + li;
        if (fabs(d2) > fmax(tau, RHO1 * (hypot(Sf.r, Sf.i) + fabs(lj) * hypot(F.r, F.i)))) {
            E21 = cscale(num, 1.0 / d2);
            const double a = E21.r * E21.r + E21.i * E21.i;
            if (a > emax2) {
                emax2 = a;
                wloc = (unsigned long long)i | ((unsigned long long)j << 20) | (1ULL << 40);
            }
        } else {
            E21 = cscale(F, -0.5);
            close++;
        }
        Et[e] = E11.r;
        Et[mm + e] = E11.i;
        Et[2 * mm + e] = E21.r;
        Et[3 * mm + e] = E21.i;
    }
    double emax = sqrt(emax2);
    for (int o = 16; o > 0; o >>= 1) {
        const double oe = __shfl_xor_sync(0xffffffffu, emax, o);
        const unsigned long long ow = __shfl_xor_sync(0xffffffffu, wloc, o);
        if (oe > emax) { emax = oe; wloc = ow; }
        close += __shfl_xor_sync(0xffffffffu, close, o);
        rn2 += __shfl_xor_sync(0xffffffffu, rn2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        const unsigned long long old = atomicMax(&sc->emax_bits, (unsigned long long)__double_as_longlong(emax));
        if ((unsigned long long)__double_as_longlong(emax) > old) atomicExch(&sc->where, wloc);
        if (close) atomicAdd(&sc->nclose, close);
        atomicAdd(&sc->rnorm2, rn2);
    }
}

// Back to the current basis: Z' = Z B (I + E~) = Z (I + E) with
// E11 = B - I + B E~11 and E21 = conj(B) E~21 (the conjugate partners rotate
// by conj(B)); then U = [[Er + Fr, Ei + Fi], [Fi - Ei, Er - Fr]].
__global__ void refine_u_kernel(int m, const int* __restrict__ cid, const double* __restrict__ Vc,
                                const double* __restrict__ Et, double* __restrict__ U, RefineScalars* sc) {
    if (sc->done) return;
    const long long mm = (long long)m * m, ldu = 2LL * m;
    double umax = 0.0;
    for (int j = blockIdx.y; j < m; j += gridDim.y)
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const long long e = (long long)j * m + q;
        cplx E11, E21;
        const int c = cid[q];
        if (c < 0) {
            E11 = {Et[e], Et[mm + e]};
            E21 = {Et[2 * mm + e], Et[3 * mm + e]};
        } else {
            const int qc = q - c;
            E11 = {0, 0};
            E21 = {0, 0};
            if (cid[j] == c) {
                E11 = {Vc[((long long)q * KC + (j - c)) * 2] - (q == j ? 1.0 : 0.0),
                       Vc[((long long)q * KC + (j - c)) * 2 + 1]};
            }
            (void)qc;
            for (int a = c; a < m && cid[a] == c; a++) {
                // B[q][a] = V_C[q - c][a - c] (row q of the cluster's V)
                const cplx b = {Vc[((long long)q * KC + (a - c)) * 2], Vc[((long long)q * KC + (a - c)) * 2 + 1]};
                const long long ea = (long long)j * m + a;
                E11 = cadd(E11, cmul(b, (cplx){Et[ea], Et[mm + ea]}));
                E21 = cadd(E21, cmul(cconj(b), (cplx){Et[2 * mm + ea], Et[3 * mm + ea]}));
            }
        }
        U[q + j * ldu] = E11.r + E21.r;
        U[q + (m + j) * ldu] = E11.i + E21.i;
        U[(m + q) + j * ldu] = E21.i - E11.i;
        U[(m + q) + (m + j) * ldu] = E11.r - E21.r;
        umax = fmax(umax, fmax(fmax(fabs(E11.r + E21.r), fabs(E11.i + E21.i)),
                               fmax(fabs(E21.i - E11.i), fabs(E11.r - E21.r))));
    }
    for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
    if ((threadIdx.x & 31) == 0 && umax > 0.0)
        atomicMax(&sc->umax_bits, (unsigned long long)__double_as_longlong(umax));
}

__global__ void refine_reset_kernel(RefineScalars* sc) {
    if (threadIdx.x == 0 && !sc->done) {
        sc->emax_bits = 0ULL;
        sc->nclose = 0u;
        sc->rnorm2 = 0.0;
        sc->where = 0ULL;
        sc->umax_bits = 0ULL;
    }
}

__global__ void lmax_kernel(int m, const double* __restrict__ lt, double* __restrict__ out,
                            const int* __restrict__ skip) {
    __shared__ double red[32];
    if (*skip) return;
    double v = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) v = fmax(v, fabs(lt[i]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) r = fmax(r, red[w]);
        *out = r;
    }
}

// The loop's state at the start of a refinement.
__global__ void refine_init_kernel(RefineScalars* sc) {
    if (threadIdx.x == 0) {
        sc->done = 0;
        sc->su = 8;
        sc->hist = RefineInfo{};
    }
}

// After the corrections of iteration it: the update's digit slices (M + M U
// with |U| <= umax needs a relative error of about 2^-62 / umax: entries of M
// ~ n^-1/2, rows of length n, so fewer slices serve once the corrections are
// small) and the iteration's record.
__global__ void refine_su_kernel(RefineScalars* sc, int it, int sl) {
    if (threadIdx.x != 0 || sc->done) return;
    const double umax = __longlong_as_double((long long)sc->umax_bits);
    int su = 8;
    if (umax > 0.0) {
        su = (int)ceil((62.0 + log2(umax)) / 7.0);
        su = su < 3 ? 3 : (su > 8 ? 8 : su);
    }
    sc->su = su;
    if (it < 8) {
        sc->hist.emax[it] = __longlong_as_double((long long)sc->emax_bits);
        sc->hist.nclose[it] = (int)sc->nclose;
        sc->hist.rnorm[it] = sqrt(sc->rnorm2);
        sc->hist.where[it] = (long long)sc->where;
        sc->hist.slices[it] = sl;
        sc->hist.uslices[it] = su;
    }
}

// End of iteration it: the next iteration would move the vectors by about
// emax^2, so the loop stops once emax is below 1e-8 (the FP64 level).
__global__ void refine_decide_kernel(RefineScalars* sc, int it) {
    if (threadIdx.x != 0 || sc->done) return;
    sc->hist.iterations = it + 1;
    if (__longlong_as_double((long long)sc->emax_bits) < 1e-8) sc->done = 1;
}

// 2-D grid for the m x m element kernels: x over i (256 threads a block), y
// over j, at most 8192 blocks
inline dim3 grid2(int m) {
    const int gx = (m + 255) / 256;
    int gy = 8192 / (gx > 0 ? gx : 1);
    if (gy > m) gy = m;
    if (gy < 1) gy = 1;
    if (gy > 65535) gy = 65535;
    return dim3((unsigned)(gx > 0 ? gx : 1), (unsigned)gy);
}


struct RefineWs {
    double *S, *Wg, *AM, *T, *U, *lt, *Vc;
    int *close, *cid, *nbig;
    RefineScalars* sc;
    // digit-slice buffers: S (once per refinement), the columns of M (Wg, AM,
    // T), the columns of AM and then of U (T, then the update), the rows of M
    // (the update)
    void *oz_s, *oz_mc, *oz_amu, *oz_mr;
    size_t oz_bytes;
};

RefineWs carve_refine(Carve& cv, int n) {
    RefineWs w{};
    const size_t nn = (size_t)n * n;
    w.S = cv.take<double>(nn);
    w.Wg = cv.take<double>(nn);
    w.AM = cv.take<double>(nn);
    w.T = cv.take<double>(nn);
    w.U = cv.take<double>(nn);
    w.lt = cv.take<double>((size_t)n);
    w.Vc = cv.take<double>((size_t)n * KC * 2);
    w.close = cv.take<int>((size_t)n);
    w.cid = cv.take<int>((size_t)n);
    w.nbig = cv.take<int>(4);
    w.sc = cv.take<RefineScalars>(1);
    w.oz_bytes = ozaki_operand_ws(n, n);
    w.oz_s = cv.take<char>(w.oz_bytes);
    w.oz_mc = cv.take<char>(w.oz_bytes);
    w.oz_amu = cv.take<char>(w.oz_bytes);
    w.oz_mr = cv.take<char>(w.oz_bytes);
    return w;
}

}  // namespace

size_t refine_ws(int n) {
    Carve cv(nullptr, ~size_t(0));
    carve_refine(cv, n);
    return cv.off + 256;
}

namespace {
// The iteration record of a refinement the device drives reaches the host in
// stream order through one pinned buffer (allocated at the first refinement
// that is not being captured into a graph; a captured one before it keeps no
// record).
struct StatsCopy {
    RefineInfo* pinned = nullptr;
    RefineInfo* target = nullptr;
    bool pending = false;
};
StatsCopy& stats_copy() {
    static StatsCopy c;
    return c;
}

int refine_stats_enqueue(cudaStream_t st, const RefineInfo* d_hist, RefineInfo* target) {
    StatsCopy& c = stats_copy();
    if (!c.pinned) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (const cudaError_t e = cudaStreamIsCapturing(st, &cs)) return cuda_fail(e);
        if (cs != cudaStreamCaptureStatusNone) return 0;
        void* p = nullptr;
        if (cudaMallocHost(&p, sizeof(RefineInfo)) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        c.pinned = static_cast<RefineInfo*>(p);
    }
    if (const cudaError_t e = cudaMemcpyAsync(c.pinned, d_hist, sizeof(RefineInfo), cudaMemcpyDeviceToHost, st))
        return cuda_fail(e);
    c.target = target;
    c.pending = true;
    return 0;
}
}  // namespace

void refine_stats_flush() {
    StatsCopy& c = stats_copy();
    if (c.pending && c.target && c.pinned) *c.target = *c.pinned;
    c.pending = false;
}

void refine_stats_discard() { stats_copy().pending = false; }

int refine(cudaStream_t st, int n, const double* A, int lda, double* lambda, double* M, int maxit, void* ws,
           size_t ws_bytes, int* status, RefineInfo* info, double rho) {
    if (n % 2 || n < 2) return SKEW_ERR_UNSUPPORTED;
    const int m = n / 2;
    Carve cv(ws, ws_bytes);
    RefineWs w = carve_refine(cv, n);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    {
        KtScope kt(st, KT_REFINE_AUX);
        skew_full_kernel<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, st>>>(n, A, lda, w.S);
    }
    count_launch();
    if (info) {
        refine_stats_discard();
        *info = RefineInfo{};
    }
    struct KindScope {  // products of this loop are timed as their own kind
        KindScope() { g_kt_ozaki_kind = KT_OZAKI_REFINE; }
        ~KindScope() { g_kt_ozaki_kind = KT_OZAKI; }
    } kind_scope;
    // The loop's decisions (tau from the largest Rayleigh quotient, the
    // update's digit slices, the stop) are taken on the device, and once the
    // loop has stopped the remaining launches return at once: no host round
    // trip, so the solve stays asynchronous and graph-capturable.  With
    // kernel timing on, the host reads the update's slice count before
    // launching the update (each timed launch records its work) and stops
    // launching when the device does; both paths take the same decisions.
    const bool host_driven = kt_enabled();
    const int* skip = &w.sc->done;
    refine_init_kernel<<<1, 32, 0, st>>>(w.sc);
    count_launch();
    const long long ldn = n;
    // row r of S is minus column r of S (skew), read contiguously
    OzOperand os{}, omc{}, oam{}, ou{}, omr{};
    int rc = ozaki_split(st, n, n, w.S, ldn, 1, -1.0, 0, w.oz_s, w.oz_bytes, &os);
    if (rc) return rc;
    for (int it = 0; it < maxit; it++) {
        // The Gram and projection products keep all eight digit slices: an
        // error delta in Wg or T enters E_ij as delta / (l_j - l_i), and dense
        // spectra have gaps far below any bound on the correction, so a
        // cheaper product stalls the iteration instead of speeding it up.
        const int sl = 8;
        // Wg = M^T M (symmetric), AM = S M, T = M^T (S M) (skew): FP64-accurate
        // tensor-core products, Wg and T on their lower triangle; the column
        // slices of M serve all three
        rc = ozaki_split(st, n, n, M, ldn, 1, 1.0, 0, w.oz_mc, w.oz_bytes, &omc, skip);
        if (rc) return rc;
        rc = ozaki_gemm_pre(st, omc, omc, 1.0, 0.0, w.Wg, ldn, status, sl, 1, 1, nullptr, 0, skip);
        if (rc) return rc;
        rc = ozaki_gemm_pre(st, os, omc, 1.0, 0.0, w.AM, ldn, status, sl, 0, 1, nullptr, 0, skip);
        if (rc) return rc;
        rc = ozaki_split(st, n, n, w.AM, ldn, 1, 1.0, 0, w.oz_amu, w.oz_bytes, &oam, skip);
        if (rc) return rc;
        rc = ozaki_gemm_pre(st, omc, oam, 1.0, 0.0, w.T, ldn, status, sl, 1, 1, nullptr, 0, skip);
        if (rc) return rc;
        {
            KtScope kt(st, KT_REFINE_AUX);
            refine_lambda_kernel<<<(m + 127) / 128, 128, 0, st>>>(m, n, w.Wg, w.T, w.lt, skip);
            refine_reset_kernel<<<1, 32, 0, st>>>(w.sc);
            lmax_kernel<<<1, 1024, 0, st>>>(m, w.lt, &w.sc->lmax, skip);
            refine_close_kernel<<<(m + 127) / 128, 128, 0, st>>>(m, n, w.Wg, w.T, w.lt, w.sc, rho, w.close);
            refine_rr_kernel<<<m, 32, 0, st>>>(m, n, w.Wg, w.T, w.close, w.lt, w.cid, w.Vc, w.nbig, skip);
            // E~ lives in the AM buffer (free once T is formed)
            refine_etilde_kernel<<<grid2(m), 256, 0, st>>>(m, n, w.Wg, w.T, w.lt, w.cid, w.Vc, w.AM, w.sc);
            refine_u_kernel<<<grid2(m), 256, 0, st>>>(m, w.cid, w.Vc, w.AM, w.U, w.sc);
            refine_su_kernel<<<1, 32, 0, st>>>(w.sc, it, sl);
        }
        count_launch(8);
        // M <- M + M U with the device's slice count (read by the kernel), or
        // with the host's copy of it when the launch is timed
        int su = 8;
        const int* su_dev = &w.sc->su;
        bool last = false;
        if (host_driven) {
            RefineScalars h{};
            if (const cudaError_t e = cudaMemcpyAsync(&h, w.sc, sizeof(h), cudaMemcpyDeviceToHost, st))
                return cuda_fail(e);
            if (const cudaError_t e = cudaStreamSynchronize(st)) return cuda_fail(e);
            if (h.done) break;
            su = h.su;
            su_dev = nullptr;
            double emax;
            std::memcpy(&emax, &h.emax_bits, sizeof(double));
            last = emax < 1e-8;  // the device's stop rule (refine_decide_kernel)
        }
        // the product reads M's digit slices, taken before C is written
        rc = ozaki_split(st, n, n, M, 1, ldn, 1.0, 0, w.oz_mr, w.oz_bytes, &omr, skip);
        if (rc) return rc;
        rc = ozaki_split(st, n, n, w.U, 2LL * m, 1, 1.0, 0, w.oz_amu, w.oz_bytes, &ou, skip);
        if (rc) return rc;
        rc = ozaki_gemm_pre(st, omr, ou, 1.0, 1.0, M, ldn, status, su, 0, 1, nullptr, 0, skip, su_dev);
        if (rc) return rc;
        // lt is left unchanged once the loop has stopped, so the copy may run
        if (const cudaError_t e = cudaMemcpyAsync(lambda, w.lt, sizeof(double) * m, cudaMemcpyDeviceToDevice, st))
            return cuda_fail(e);
        refine_decide_kernel<<<1, 32, 0, st>>>(w.sc, it);
        count_launch();
        if (last) break;
    }
    if (info) {
        // the iteration record: read now when the host drives the loop,
        // otherwise copied in stream order for refine_stats_flush()
        if (host_driven) {
            if (const cudaError_t e = cudaMemcpyAsync(info, &w.sc->hist, sizeof(RefineInfo), cudaMemcpyDeviceToHost, st))
                return cuda_fail(e);
            if (const cudaError_t e = cudaStreamSynchronize(st)) return cuda_fail(e);
        } else {
            rc = refine_stats_enqueue(st, &w.sc->hist, info);
            if (rc) return rc;
        }
    }
    return cuda_ok(cudaGetLastError());
}

}  // namespace sk
