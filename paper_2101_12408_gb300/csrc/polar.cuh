// 3x3 polar decomposition F = R S and the fixed-corotated solid.
//
// Written from the mathematics: the eigenvectors V of F^T F by cyclic Jacobi
// rotations, singular values sorted descending, U's columns u1 = F v1/|F v1|,
// u2 by Gram-Schmidt of F v2, u3 = u1 x u2 (so U and V are rotations and the
// smallest singular value carries the sign of det F, the "polar SVD"), R = U V^T.
// (tr S I - S)^-1 = V diag(1/(s2+s3), 1/(s1+s3), 1/(s1+s2)) V^T is returned for
// the rotation differential dR = R [w]x, (tr S I - S) w = axial(R^T dF - dF^T R).
// Fixed corotated (paper section "Constitutive Models"):
//   psi = mu sum (s_a - 1)^2 + lambda/2 (J - 1)^2,  P = 2 mu (F - R) + lambda (J - 1) cof F.
#pragma once
#include "common.cuh"

namespace mpm {

template <typename R>
__device__ __forceinline__ void jacobi_rot(R* A, R* V, int p, int q) {
    R apq = A[3 * p + q];
    if (apq == R(0)) return;
    R theta = (A[3 * q + q] - A[3 * p + p]) / (R(2) * apq);
    R t;
    if (fabs(theta) > R(1e12)) t = R(0.5) / theta;
    else t = copysign(R(1), theta) / (fabs(theta) + sqrt(theta * theta + R(1)));
    R c = R(1) / sqrt(t * t + R(1));
    R s = t * c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - s * akq;
        A[3 * k + q] = s * akp + c * akq;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - s * aqk;
        A[3 * q + k] = s * apk + c * aqk;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - s * vkq;
        V[3 * k + q] = s * vkp + c * vkq;
    }
}

template <typename R>
__device__ __forceinline__ void swap_cols(R* V, R* lam, int a, int b) {
    R t = lam[a];
    lam[a] = lam[b];
    lam[b] = t;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R u = V[3 * k + a];
        V[3 * k + a] = V[3 * k + b];
        V[3 * k + b] = -u;   // keep det V = +1
    }
}

// Signed SVD F = U diag(sig) V^T with U, V rotations (u[k] is U's column k,
// V row-major), singular values descending in magnitude, the last one carrying
// the sign of det F.
template <typename R>
__device__ void svd3(const R* F, R (*u)[3], R* V, R* sig) {
    R A[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? R(1) : R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
    const R eps = sizeof(R) == 4 ? R(1e-7) : R(1e-16);
    for (int sweep = 0; sweep < 12; ++sweep) {
        R off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        R dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= eps * eps * dia) break;
        jacobi_rot(A, V, 0, 1);
        jacobi_rot(A, V, 0, 2);
        jacobi_rot(A, V, 1, 2);
    }
    R lam[3] = {A[0], A[4], A[8]};
    if (lam[0] < lam[1]) swap_cols(V, lam, 0, 1);
    if (lam[0] < lam[2]) swap_cols(V, lam, 0, 2);
    if (lam[1] < lam[2]) swap_cols(V, lam, 1, 2);
    R Fv[3][3];   // F v_k
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) Fv[k][i] = F[3 * i] * V[k] + F[3 * i + 1] * V[3 + k] + F[3 * i + 2] * V[6 + k];
    R n1 = sqrt(Fv[0][0] * Fv[0][0] + Fv[0][1] * Fv[0][1] + Fv[0][2] * Fv[0][2]);
    if (n1 > R(1e-30)) {
        for (int i = 0; i < 3; ++i) u[0][i] = Fv[0][i] / n1;
    } else {
        u[0][0] = 1; u[0][1] = 0; u[0][2] = 0;
    }
    R d = u[0][0] * Fv[1][0] + u[0][1] * Fv[1][1] + u[0][2] * Fv[1][2];
    R w2[3] = {Fv[1][0] - d * u[0][0], Fv[1][1] - d * u[0][1], Fv[1][2] - d * u[0][2]};
    R n2 = sqrt(w2[0] * w2[0] + w2[1] * w2[1] + w2[2] * w2[2]);
    if (n2 > R(1e-30) * (n1 + R(1e-30))) {
        for (int i = 0; i < 3; ++i) u[1][i] = w2[i] / n2;
    } else {
        // any unit vector orthogonal to u0
        R a[3] = {R(0), R(0), R(0)};
        int m = fabs(u[0][0]) < fabs(u[0][1]) ? (fabs(u[0][0]) < fabs(u[0][2]) ? 0 : 2) : (fabs(u[0][1]) < fabs(u[0][2]) ? 1 : 2);
        a[m] = 1;
        R dd = u[0][m];
        for (int i = 0; i < 3; ++i) a[i] -= dd * u[0][i];
        R na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int i = 0; i < 3; ++i) u[1][i] = a[i] / na;
    }
    u[2][0] = u[0][1] * u[1][2] - u[0][2] * u[1][1];
    u[2][1] = u[0][2] * u[1][0] - u[0][0] * u[1][2];
    u[2][2] = u[0][0] * u[1][1] - u[0][1] * u[1][0];
#pragma unroll
    for (int k = 0; k < 3; ++k) sig[k] = u[k][0] * Fv[k][0] + u[k][1] * Fv[k][1] + u[k][2] * Fv[k][2];
}

// F -> rotation Rm, (tr S I - S)^-1 as symmetric 6 (xx yy zz xy xz yz), signed singular values
template <typename R>
__device__ void polar3(const R* F, R* Rm, R* Kinv, R* sig) {
    R u[3][3], V[9];
    svd3<R>(F, u, V, sig);
    // R = U V^T : R_ij = sum_k u[k][i] V[j][k]
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Rm[3 * i + j] = u[0][i] * V[3 * j] + u[1][i] * V[3 * j + 1] + u[2][i] * V[3 * j + 2];
    R e[3] = {sig[1] + sig[2], sig[0] + sig[2], sig[0] + sig[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) e[k] = R(1) / (fabs(e[k]) > R(1e-12) ? e[k] : copysign(R(1e-12), e[k]));
    // Kinv = V diag(e) V^T
    Kinv[0] = V[0] * V[0] * e[0] + V[1] * V[1] * e[1] + V[2] * V[2] * e[2];
    Kinv[1] = V[3] * V[3] * e[0] + V[4] * V[4] * e[1] + V[5] * V[5] * e[2];
    Kinv[2] = V[6] * V[6] * e[0] + V[7] * V[7] * e[1] + V[8] * V[8] * e[2];
    Kinv[3] = V[0] * V[3] * e[0] + V[1] * V[4] * e[1] + V[2] * V[5] * e[2];
    Kinv[4] = V[0] * V[6] * e[0] + V[1] * V[7] * e[1] + V[2] * V[8] * e[2];
    Kinv[5] = V[3] * V[6] * e[0] + V[4] * V[7] * e[1] + V[5] * V[8] * e[2];
}

template <typename R>
__device__ __forceinline__ R fcr_psi(const R* F, R mu, R lam) {
    R Rm[9], K[6], s[3];
    polar3<R>(F, Rm, K, s);
    R J = det3<R>(F);
    return mu * ((s[0] - 1) * (s[0] - 1) + (s[1] - 1) * (s[1] - 1) + (s[2] - 1) * (s[2] - 1)) +
           R(0.5) * lam * (J - 1) * (J - 1);
}

// dP = 2 mu (dF - dR) + lambda (cof F : dF) cof F + lambda (J - 1) dcof(F)[dF]
template <typename R>
__device__ __forceinline__ void fcr_dP(const R* F, const R* Rm, const R* K, R mu, R lam, const R* dF, R* dP) {
    R X[9];   // R^T dF
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X[3 * i + j] = Rm[i] * dF[j] + Rm[3 + i] * dF[3 + j] + Rm[6 + i] * dF[6 + j];
    R b[3] = {X[7] - X[5], X[2] - X[6], X[3] - X[1]};   // axial(X - X^T)
    R w[3] = {K[0] * b[0] + K[3] * b[1] + K[4] * b[2], K[3] * b[0] + K[1] * b[1] + K[5] * b[2],
              K[4] * b[0] + K[5] * b[1] + K[2] * b[2]};
    R W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    R dR[9];
    matmul3<R>(Rm, W, dR);
    R C[9], dC[9];
    cofactor<R>(F, C);
    dcofactor<R>(F, dF, dC);
    R J = det3<R>(F);
    R cdf = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) cdf += C[k] * dF[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) dP[k] = R(2) * mu * (dF[k] - dR[k]) + lam * cdf * C[k] + lam * (J - 1) * dC[k];
}

}  // namespace mpm
