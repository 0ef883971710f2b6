// Cyclic Jacobi eigensolver of a small symmetric matrix held in shared memory, run by one CTA.
//
// Every round applies m/2 disjoint plane rotations chosen by round-robin pairing (position 0
// fixed, the others rotating), each the symmetric 2 x 2 Schur rotation that annihilates its
// off-diagonal pair: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1 / sqrt(1 + t^2), s = t c; A := J^T A J and Q := Q J.  Sweeps (m - 1 rounds each) until the
// off-diagonal mass is at most 1e-32 of the total, or max_sweeps.
#pragma once

namespace oz {

struct JacobiScratch {
  double* cs;   // >= (m + 1) / 2
  double* sn;   // >= (m + 1) / 2
  int* pp;      // >= (m + 1) / 2
  int* qq;      // >= (m + 1) / 2
  double* red;  // >= 2 * blockDim.x / 32
  int* stop;    // 1
};

__device__ __forceinline__ double jacobi_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A: m x m symmetric (element (i, j) at A[i * lda + j]), overwritten by its diagonalised form;
// Q (same layout) receives the eigenvectors as columns: the rotations are accumulated onto the
// identity, or onto the given Q when init_q is false (then Q^T (original) Q = A on entry, and the
// eigenvectors of the original matrix come out).  With negl > 0 an off-diagonal element at most
// negl (|a_pp| + |a_qq|) is set to zero instead of rotated (the classical threshold of cyclic
// Jacobi: below the rounding of its diagonal pair it cannot change the eigenvalues).  Every thread of
// the CTA must call it.  Returns the number of sweeps taken, or -1 if max_sweeps did not converge.
__device__ inline int jacobi_smem(double* A, double* Q, int lda, int m, JacobiScratch w, int max_sweeps,
                                  bool init_q = true, double negl = 0.0) {
  const int tid = threadIdx.x, nth = blockDim.x, nwarp = (nth + 31) / 32;
  if (init_q)
    for (int idx = tid; idx < m * m; idx += nth) {
      const int i = idx / m, j = idx % m;
      Q[i * lda + j] = i == j ? 1.0 : 0.0;
    }
  __syncthreads();
  const int mm = m + (m & 1), npair = mm / 2;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < m * m; idx += nth) {
      const int i = idx / m, j = idx % m;
      const double a2 = A[i * lda + j] * A[i * lda + j];
      tot += a2;
      if (i != j) off += a2;
    }
    off = jacobi_warp_sum(off);
    tot = jacobi_warp_sum(tot);
    if ((tid & 31) == 0) {
      w.red[2 * (tid >> 5)] = off;
      w.red[2 * (tid >> 5) + 1] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, t = 0.0;
      for (int k = 0; k < nwarp; ++k) {
        o += w.red[2 * k];
        t += w.red[2 * k + 1];
      }
      *w.stop = (o <= 1e-32 * t) ? 1 : 0;
    }
    __syncthreads();
    if (*w.stop) return sweep;
    if (sweep == max_sweeps) break;
    for (int r = 0; r < mm - 1; ++r) {
      for (int k = tid; k < npair; k += nth) {
        const int a = k == 0 ? 0 : 1 + (k - 1 + r) % (mm - 1);
        const int bpos = mm - 1 - k;
        const int b = bpos == 0 ? 0 : 1 + (bpos - 1 + r) % (mm - 1);
        const int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < m && negl > 0.0 && A[p * lda + q] != 0.0 &&
            fabs(A[p * lda + q]) <= negl * (fabs(A[p * lda + p]) + fabs(A[q * lda + q]))) {
          A[p * lda + q] = 0.0;  // each pair is owned by one thread in this round
          A[q * lda + p] = 0.0;
        } else if (q < m && A[p * lda + q] != 0.0) {
          const double apq = A[p * lda + q];
          const double tau = (A[q * lda + q] - A[p * lda + p]) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        w.cs[k] = c;
        w.sn[k] = s;
        w.pp[k] = p;
        w.qq[k] = q < m ? q : p;  // a dummy partner turns into the identity
      }
      __syncthreads();
      for (int idx = tid; idx < npair * m; idx += nth) {  // A := A J, Q := Q J (columns p, q)
        const int k = idx / m, row = idx % m;
        const double s = w.sn[k];
        if (s == 0.0) continue;
        const int p = w.pp[k], q = w.qq[k];
        const double c = w.cs[k];
        const double ap = A[row * lda + p], aq = A[row * lda + q];
        A[row * lda + p] = c * ap - s * aq;
        A[row * lda + q] = s * ap + c * aq;
        const double vp = Q[row * lda + p], vq = Q[row * lda + q];
        Q[row * lda + p] = c * vp - s * vq;
        Q[row * lda + q] = s * vp + c * vq;
      }
      __syncthreads();
      for (int idx = tid; idx < npair * m; idx += nth) {  // A := J^T A (rows p, q)
        const int k = idx / m, col = idx % m;
        const double s = w.sn[k];
        if (s == 0.0) continue;
        const int p = w.pp[k], q = w.qq[k];
        const double c = w.cs[k];
        const double ap = A[p * lda + col], aq = A[q * lda + col];
        A[p * lda + col] = c * ap - s * aq;
        A[q * lda + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int k = tid; k < npair; k += nth)
        if (w.sn[k] != 0.0) {
          A[w.pp[k] * lda + w.qq[k]] = 0.0;
          A[w.qq[k] * lda + w.pp[k]] = 0.0;
        }
      __syncthreads();
    }
  }
  return -1;
}

// order[0..m) = indices of the diagonal of A sorted ascending (descending = false) or descending,
// ties by index (insertion sort by one thread; m is small).
__device__ inline void jacobi_order(const double* A, int lda, int m, bool descending, int* order) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 1; i < m; ++i) {
      const int v = order[i];
      int j = i - 1;
      while (j >= 0 && (descending ? A[order[j] * lda + order[j]] < A[v * lda + v]
                                   : A[order[j] * lda + order[j]] > A[v * lda + v])) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = v;
    }
  }
  __syncthreads();
}

}  // namespace oz
