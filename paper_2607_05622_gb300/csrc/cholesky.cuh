// Cholesky-factorised J/K (Eqs. cdfact, cdj, cdknonsym): the pivoted
// incomplete Cholesky factor B of the ERI matrix, with its columns evaluated
// by the same quartet kernels as the direct build, and J and K of densities
// given as factors D[q] = U[q] V[q]^T read off B by dense contractions.
// Included by context.cu only (it uses the context internals).
#pragma once

namespace ltjk {
namespace {

// d[mu*N+nu] = (mu nu|mu nu) from the diagonal shell-quartet blocks (ab|ab),
// block k at blocks + off[k], layout [na][nb][na][nb]; both (mu,nu) orders.
__global__ void cd_diag_scatter(const double *__restrict__ blocks, const long long *__restrict__ off,
                                const int4 *__restrict__ pairs, int npairs, int N, double *__restrict__ d) {
  for (int k = blockIdx.x; k < npairs; k += gridDim.x) {
    const int4 P = pairs[k];  // a0, na, b0, nb
    const double *blk = blocks + off[k];
    for (int e = threadIdx.x; e < P.y * P.w; e += blockDim.x) {
      const int i = e / P.w, j = e % P.w;
      const double v = blk[(size_t)(i * P.w + j) * (P.y * P.w) + i * P.w + j];
      d[(size_t)(P.x + i) * N + P.z + j] = v;
      d[(size_t)(P.z + j) * N + P.x + i] = v;
    }
  }
}

// Columns of the pivot shell pair (s,t): blocks (ab|st) for every pair ab,
// layout [na][nb][ns][nt]; column c = k*nt + l holds (mu nu|s_k t_l) for all
// ordered (mu, nu), written into cols[c][mu*N + nu].
__global__ void cd_col_scatter(const double *__restrict__ blocks, const long long *__restrict__ off,
                               const int4 *__restrict__ pairs, int npairs, int N, int nst,
                               double *__restrict__ cols) {
  const size_t NN = (size_t)N * N;
  for (int k = blockIdx.x; k < npairs; k += gridDim.x) {
    const int4 P = pairs[k];
    const double *blk = blocks + off[k];
    const int n = P.y * P.w * nst;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int c = e % nst, ij = e / nst, i = ij / P.w, j = ij % P.w;
      const double v = blk[e];
      cols[c * NN + (size_t)(P.x + i) * N + P.z + j] = v;
      cols[c * NN + (size_t)(P.z + j) * N + P.x + i] = v;
    }
  }
}

// Largest residual diagonal over the unique pairs mu >= nu (lowest index on
// ties): one CTA of 1024 threads; out_val[0], out_idx[0].
__global__ void cd_argmax(const double *__restrict__ d, int N, double *out_val, int *out_idx) {
  __shared__ double sv[32];
  __shared__ int si[32];
  double best = -1.0;
  int bi = 0x7fffffff;
  const int NN = N * N;
  for (int r = threadIdx.x; r < NN; r += blockDim.x) {
    const int mu = r / N, nu = r - mu * N;
    if (nu > mu) continue;
    const double v = d[r];
    if (v > best || (v == best && r < bi)) {
      best = v;
      bi = r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sv[warp] = best;
    si[warp] = bi;
  }
  __syncthreads();
  if (warp == 0) {
    best = lane < (int)(blockDim.x >> 5) ? sv[lane] : -1.0;
    bi = lane < (int)(blockDim.x >> 5) ? si[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      out_val[0] = best;
      out_idx[0] = bi;
    }
  }
}

// One Cholesky step at pivot p: L[r] = (col[r] - sum_{k<nvec} B[k][r] B[k][p])
// * inv_sqrt_dp and d[r] -= L[r]^2 for every ordered pair r; d[p] = 0.
__global__ void cd_step(const double *__restrict__ col, const double *__restrict__ B, int nvec, int p,
                        double inv_sqrt_dp, double *__restrict__ L, double *__restrict__ d, size_t NN) {
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < NN; r += (size_t)gridDim.x * blockDim.x) {
    double s0 = col[r], s1 = 0.0;
    int k = 0;
    for (; k + 1 < nvec; k += 2) {  // two independent chains
      s0 = fma(-__ldg(B + (size_t)k * NN + r), __ldg(B + (size_t)k * NN + p), s0);
      s1 = fma(-__ldg(B + (size_t)(k + 1) * NN + r), __ldg(B + (size_t)(k + 1) * NN + p), s1);
    }
    if (k < nvec) s0 = fma(-__ldg(B + (size_t)k * NN + r), __ldg(B + (size_t)k * NN + p), s0);
    const double l = (s0 + s1) * inv_sqrt_dp;
    L[r] = l;
    d[r] = r == (size_t)p ? 0.0 : fma(-l, l, d[r]);
  }
}

// C[m][n] = sum_k A[m][k] Bm[k][n] (+= when ACC), row-major, 16 x 16 tiles with
// the M tiles on grid x (no 65535 limit); FP64, one output per thread.  The
// FP64 FMA pipe (2 per clock per SM) is slower than the shared-memory operand
// path here, so this plain tiling already runs at the pipe's rate.
template <bool ACC>
__global__ void cd_gemm(const double *__restrict__ A, const double *__restrict__ Bm, double *__restrict__ C,
                        long long M, int Nn, int Kd, int lda, int ldb, int ldc) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long m0 = (long long)blockIdx.x * 16;
  const int n0 = blockIdx.y * 16;
  double acc = 0.0;
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    As[ty][tx] = (m0 + ty < M && k0 + tx < Kd) ? A[(size_t)(m0 + ty) * lda + k0 + tx] : 0.0;
    Bs[ty][tx] = (k0 + ty < Kd && n0 + tx < Nn) ? Bm[(size_t)(k0 + ty) * ldb + n0 + tx] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (m0 + ty < M && n0 + tx < Nn) {
    double *c = C + (size_t)(m0 + ty) * ldc + n0 + tx;
    *c = ACC ? *c + acc : acc;
  }
}

// K[mu][nu] += sum_{Q in chunk} sum_m BU[Q][mu][m] BV[Q][nu][m] (Eq. cdknonsym):
// 16 x 16 output tiles, the auxiliary index split over grid z (FP64 atomics).
__global__ void cd_k_contract(const double *__restrict__ BU, const double *__restrict__ BV, int naux, int N,
                              int rank, int qchunk, double *__restrict__ K) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int mu0 = blockIdx.x * 16, nu0 = blockIdx.y * 16;
  const int q0 = blockIdx.z * qchunk, q1 = min(naux, q0 + qchunk);
  const size_t qs = (size_t)N * rank;
  double acc = 0.0;
  for (int Q = q0; Q < q1; ++Q) {
    const double *U = BU + Q * qs, *V = BV + Q * qs;
    for (int m0 = 0; m0 < rank; m0 += 16) {
      As[ty][tx] = (mu0 + ty < N && m0 + tx < rank) ? U[(size_t)(mu0 + ty) * rank + m0 + tx] : 0.0;
      Bs[ty][tx] = (nu0 + ty < N && m0 + tx < rank) ? V[(size_t)(nu0 + ty) * rank + m0 + tx] : 0.0;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[tx][k], acc);
      __syncthreads();
    }
  }
  if (mu0 + ty < N && nu0 + tx < N) atomicAdd(K + (size_t)(mu0 + ty) * N + nu0 + tx, acc);
}

// gamma[Q] = sum_{mu, m} BU[Q][mu][m] V[mu][m] = sum_{mu ka} B_Q[mu][ka] D[ka][mu],
// which is <B_Q, D> of Eq. cdj because every B_Q is symmetric: one CTA per Q.
__global__ void cd_gamma(const double *__restrict__ BU, const double *__restrict__ V, int naux, size_t per,
                         double *__restrict__ gamma) {
  __shared__ double red[32];
  for (int Q = blockIdx.x; Q < naux; Q += gridDim.x) {
    const double *u = BU + Q * per;
    double s = 0.0;
    for (size_t e = threadIdx.x; e < per; e += blockDim.x) s = fma(u[e], V[e], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) gamma[Q] = s;
    }
    __syncthreads();
  }
}

// C = A B'^T in double-float on the FP32 pipe: A [M][lda] and B' [Nc][ldb] are
// FP64, both with the contracted index k contiguous; each 256-thread CTA owns a
// 64 x 64 tile of C (4 x 4 per thread) and the k range [z kchunk, (z+1) kchunk)
// of its grid slice z.  Operand tiles are split to float pairs when staged in
// shared memory; products and sums are double-float (~2^-44 per operation).
// Epilogue PERM (one k slice): row i = Q*N + mu, column c = q*r + m of the
// product B_flat V^T is stored at C[q][mu][Q][m] (the [mu][(Q,m)] layout that
// makes (Q, m) one contiguous index of the exchange contraction).  Epilogue
// ATOMIC: FP64 atomicAdd of the tile into C[i*ldc + c] (split-k partial sums).
// Epilogue ATOMIC_K: column c = j*N + nu of a chunk of densities stacked along
// the columns goes to C[j][i][nu] (the exchange matrices of the chunk).
constexpr int kEpiPerm = 0, kEpiAtomic = 1, kEpiAtomicK = 2;
struct PermShape {
  int N, naux, r;
};
template <int EPI>
__global__ void __launch_bounds__(256) cd_gemm_nt_df(const double *__restrict__ A, int lda,
                                                     const double *__restrict__ Bt, int ldb,
                                                     double *__restrict__ C, int ldc, long long M, int Nc,
                                                     long long Kd, long long kchunk, PermShape ps) {
  __shared__ float2 As[16][64 + 4];  // [k][row]
  __shared__ float2 Bs[16][64 + 4];  // [k][col]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * 64;
  const int n0 = blockIdx.y * 64;
  const long long kz0 = (long long)blockIdx.z * kchunk, kz1 = min(Kd, kz0 + kchunk);
  dflt acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero_real<dflt>();
  for (long long k0 = kz0; k0 < kz1; k0 += 16) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {  // 64 rows x 16 k of each operand, coalesced along k
      const int e = tid + 256 * t, row = e >> 4, kk = e & 15;
      const bool kin = k0 + kk < kz1;
      const double va = (m0 + row < M && kin) ? A[(size_t)(m0 + row) * lda + k0 + kk] : 0.0;
      const double vb = (n0 + row < Nc && kin) ? Bt[(size_t)(n0 + row) * ldb + k0 + kk] : 0.0;
      float h, l;
      d2f_split(va, h, l);
      As[kk][row] = make_float2(h, l);
      d2f_split(vb, h, l);
      Bs[kk][row] = make_float2(h, l);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      dflt a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 fa = As[kk][ty * 4 + i], fb = Bs[kk][tx * 4 + i];
        a[i] = dflt(fa.x, fa.y);
        b[i] = dflt(fb.x, fb.y);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx * 4 + j;
      if (c >= Nc) continue;
      const double v = to_double(acc[i][j]);
      if (EPI == kEpiAtomic) {
        atomicAdd(C + (size_t)m * ldc + c, v);
      } else if (EPI == kEpiAtomicK) {
        const int j = c / ps.N, nu = c - j * ps.N;
        atomicAdd(C + ((size_t)j * ps.N + m) * ps.N + nu, v);
      } else {
        const long long Q = m / ps.N, mu = m - Q * ps.N;
        const int q = c / ps.r, mm = c - q * ps.r;
        C[(((size_t)q * ps.N + mu) * ps.naux + Q) * ps.r + mm] = v;
      }
    }
  }
}

// out[q*r + m][k] = V[q][k][m] for q < nq (the B' operand of B_flat V^T).
__global__ void cd_transpose_factors(const double *__restrict__ V, int nq, int N, int r,
                                     double *__restrict__ out) {
  const size_t n = (size_t)nq * N * r;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % N);
    const size_t qm = t / N;
    const int q = (int)(qm / r), m = (int)(qm % r);
    out[t] = V[((size_t)q * N + k) * r + m];
  }
}

// gamma[q][Q] = sum_{mu, m} BU_q[mu][Q][m] V[q][mu][m] with BU_q = BU + q bu_stride
// (bu_stride 0 when all densities share the left factor): one warp per (q, Q).
__global__ void cd_gamma_perm(const double *__restrict__ BU, size_t bu_stride, const double *__restrict__ V,
                              int nq, int naux, int N, int r, double *__restrict__ gamma) {
  const int lane = threadIdx.x & 31;
  for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < (long long)nq * naux;
       w += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int q = (int)(w / naux), Q = (int)(w % naux);
    double s = 0.0;
    for (int e = lane; e < N * r; e += 32) {
      const int mu = e / r, m = e - mu * r;
      s = fma(BU[q * bu_stride + ((size_t)mu * naux + Q) * r + m], V[((size_t)q * N + mu) * r + m], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) gamma[(size_t)q * naux + Q] = s;
  }
}

// U[q] = C_occ for every density q (the left factor shared by all of them).
__global__ void cd_replicate(const double *__restrict__ C, size_t n, int nq, double *__restrict__ U) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n * nq; t += (size_t)gridDim.x * blockDim.x)
    U[t] = C[t % n];
}

// The shell pair and component orientation of AO pair (mu, nu) in the
// context's canonical pair order: pair index, and the column of that pair's
// block that holds (.|mu nu).
struct PivotPair {
  int pair;    // sorted pair index of the canonical (s, t)
  int column;  // k * nt + l with k in s, l in t
};

PivotPair pivot_pair(const ltjk_ctx &c, const std::vector<int> &ao_shell, int mu, int nu) {
  const int s1 = ao_shell[mu], s2 = ao_shell[nu];
  auto it = c.pair_of.find({s1, s2});
  int t = s2, k = mu - c.sh_ao[s1], l = nu - c.sh_ao[s2];
  if (it == c.pair_of.end()) {  // (.|mu nu) = (.|nu mu): use the canonical (s2, s1)
    it = c.pair_of.find({s2, s1});
    t = s1;
    k = nu - c.sh_ao[s2];
    l = mu - c.sh_ao[s1];
  }
  return PivotPair{it->second, k * ncart(c.sh_l[t]) + l};
}

// Pair geometry (a0, na, b0, nb) of every sorted pair, for the scatter kernels.
std::vector<int4> pair_geometry(const ltjk_ctx &c) {
  std::vector<int4> g(c.npairs);
  for (int i = 0; i < c.npairs; ++i) {
    const int2 ab = c.pair_sh[i];
    g[i] = make_int4(c.sh_ao[ab.x], ncart(c.sh_l[ab.x]), c.sh_ao[ab.y], ncart(c.sh_l[ab.y]));
  }
  return g;
}

}  // namespace
}  // namespace ltjk

extern "C" {

int ltjk_cd_factor(ltjk_ctx *ctx, double delta, int max_vectors, double *B, int *naux, double *max_residual,
                   ltjk_stream stream) {
  using namespace ltjk;
  if (!ctx || !B || !naux) return set_error(LTJK_EINVAL, "cd_factor: null argument");
  if (!(delta > 0.0) || max_vectors < 1)
    return set_error(LTJK_EINVAL, "cd_factor: need delta > 0 and max_vectors >= 1");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ltjk_ctx &c = *ctx;
  const int N = c.nao;
  const size_t NN = (size_t)N * N;
  std::vector<int> ao_shell(N);
  for (int s = 0; s < c.nshells; ++s)
    for (int k = 0; k < ncart(c.sh_l[s]); ++k) ao_shell[c.sh_ao[s] + k] = s;
  const std::vector<int4> geo = pair_geometry(c);
  DevBuf d_geo, d_d, d_best, d_off, d_blocks;
  int rc;
  if ((rc = d_geo.upload(geo)) || (rc = d_d.alloc(NN * sizeof(double), st)) ||
      (rc = d_best.alloc(2 * sizeof(double), st)))
    return rc;
  // residual diagonal from the diagonal quartets (ab|ab), IEEE FP64
  {
    std::vector<std::pair<int, int>> qs;
    for (int i = 0; i < c.npairs; ++i) qs.push_back({i, i});
    long long total = 0;
    for (const int4 &g : geo) total += (long long)g.y * g.w * g.y * g.w;
    if ((rc = d_blocks.alloc((size_t)total * sizeof(double), st))) return rc;
    std::vector<long long> offs;
    if ((rc = store_blocks(c, qs, LTJK_FP64_NATIVE, offs, d_blocks.as<double>(), st))) return rc;
    if ((rc = d_off.upload(offs))) return rc;
    CUDA_TRY(cudaMemsetAsync(d_d.p, 0, NN * sizeof(double), st));
    cd_diag_scatter<<<std::min(c.npairs, num_sms() * 8), 128, 0, st>>>(
        d_blocks.as<double>(), d_off.as<long long>(), d_geo.as<int4>(), c.npairs, N, d_d.as<double>());
    CUDA_TRY(cudaGetLastError());
    g_launches += 1;
  }
  // column blocks of the pivot shell pairs, computed on first use
  std::map<int, std::unique_ptr<DevBuf>> cols;
  std::vector<std::pair<int, int>> qs(c.npairs);
  std::vector<long long> offs;
  {
    long long total = 0;  // blocks (ab|st) of every pair ab for the largest pivot pair (dd: 36)
    const int nmax = ncart(kMaxL) * ncart(kMaxL);
    for (const int4 &g : geo) total += (long long)g.y * g.w * nmax;
    if ((size_t)total * sizeof(double) > d_blocks.bytes &&
        (rc = d_blocks.alloc((size_t)total * sizeof(double), st)))
      return rc;
  }
  int nvec = 0;
  double best = 0.0;
  const int steps_grid = (int)std::min<size_t>((NN + 255) / 256, num_sms() * 16);
  for (;;) {
    cd_argmax<<<1, 1024, 0, st>>>(d_d.as<double>(), N, d_best.as<double>(),
                                  reinterpret_cast<int *>(d_best.as<double>() + 1));
    CUDA_TRY(cudaGetLastError());
    g_launches += 1;
    double hv[2];
    CUDA_TRY(cudaMemcpyAsync(hv, d_best.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    best = hv[0];
    int p;
    std::memcpy(&p, &hv[1], sizeof(int));
    if (!(best > delta) || nvec >= max_vectors) break;
    const PivotPair pv = pivot_pair(c, ao_shell, p / N, p % N);
    auto it = cols.find(pv.pair);
    if (it == cols.end()) {
      const int2 st_sh = c.pair_sh[pv.pair];
      const int nst = ncart(c.sh_l[st_sh.x]) * ncart(c.sh_l[st_sh.y]);
      for (int i = 0; i < c.npairs; ++i) qs[i] = {i, pv.pair};
      if ((rc = store_blocks(c, qs, LTJK_FP64_NATIVE, offs, d_blocks.as<double>(), st))) return rc;
      if ((rc = d_off.upload(offs))) return rc;
      auto buf = std::make_unique<DevBuf>();
      if ((rc = buf->alloc((size_t)nst * NN * sizeof(double), st))) return rc;
      cd_col_scatter<<<std::min(c.npairs, num_sms() * 8), 128, 0, st>>>(
          d_blocks.as<double>(), d_off.as<long long>(), d_geo.as<int4>(), c.npairs, N, nst, buf->as<double>());
      CUDA_TRY(cudaGetLastError());
      g_launches += 1;
      it = cols.emplace(pv.pair, std::move(buf)).first;
    }
    const double *col = it->second->as<double>() + (size_t)pv.column * NN;
    cd_step<<<steps_grid, 256, 0, st>>>(col, B, nvec, p, 1.0 / std::sqrt(best), B + (size_t)nvec * NN,
                                        d_d.as<double>(), NN);
    CUDA_TRY(cudaGetLastError());
    g_launches += 1;
    ++nvec;
  }
  CUDA_TRY(cudaStreamSynchronize(st));  // the column cache and scratch die here
  *naux = nvec;
  if (max_residual) *max_residual = best;
  return LTJK_OK;
}

int ltjk_pseudo_density_factors(ltjk_ctx *ctx, int nocc, int nvir, const double *C_occ,
                                const double *C_vir, const double *eps_occ, const double *eps_vir,
                                int npair, const double *X, int nlap, const double *t_host, double *U,
                                double *V, ltjk_stream stream) {
  using namespace ltjk;
  if (!ctx || !C_occ || !C_vir || !eps_occ || !eps_vir || !X || !t_host || !U || !V)
    return set_error(LTJK_EINVAL, "pseudo_density_factors: null argument");
  if (nocc < 1 || nvir < 1 || npair < 1 || nlap < 1 || (long long)npair * nlap > 4096)
    return set_error(LTJK_EINVAL, "pseudo_density_factors: bad sizes");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int N = ctx->nao, nq = nlap * npair;
  const size_t ny = (size_t)nq * nocc * nvir, nu = (size_t)N * nocc;
  int rc;
  if (ctx->d_t.bytes < sizeof(double) * nlap &&
      (rc = ctx->d_t.alloc(sizeof(double) * 64 * ((nlap + 63) / 64), st)))
    return rc;
  if ((rc = ctx->ensure_scratch(ny * sizeof(double), st))) return rc;
  double *Y = ctx->scratch.as<double>();
  CUDA_TRY(cudaMemcpyAsync(ctx->d_t.p, t_host, sizeof(double) * nlap, cudaMemcpyHostToDevice, st));
  // Y[q*npair+p][i][a] = exp(t_q (eps_i - eps_a)) X[p][i][a]   (Eq. scaledcoeff)
  scale_amplitudes<<<(int)std::min<size_t>((ny + 255) / 256, num_sms() * 16), 256, 0, st>>>(
      X, eps_occ, eps_vir, ctx->d_t.as<double>(), Y, nlap, npair, nocc, nvir);
  // V[q] = C_vir Y[q]^T   ([N][nvir] x [nvir][nocc])
  const dim3 thr(16, 16), g((nocc + 15) / 16, (N + 15) / 16, nq);
  gemm_f64<true><<<g, thr, 0, st>>>(C_vir, 0, Y, (long long)nocc * nvir, V, (long long)nu, N, nocc, nvir, nvir,
                                    nvir, nocc);
  cd_replicate<<<(int)std::min<size_t>((nu * nq + 255) / 256, num_sms() * 16), 256, 0, st>>>(C_occ, nu, nq, U);
  CUDA_TRY(cudaGetLastError());
  g_launches += 3;
  return LTJK_OK;
}

int ltjk_cd_jk(ltjk_ctx *ctx, int naux, const double *B, int ndens, int rank, int u_count, const double *U,
               const double *V, double *J, double *K, ltjk_stream stream) {
  using namespace ltjk;
  if (!ctx || !B || !U || !V || (!J && !K)) return set_error(LTJK_EINVAL, "cd_jk: null argument");
  if (naux < 1 || ndens < 1 || ndens > 4096 || rank < 1 || rank > ctx->nao ||
      (u_count != 1 && u_count != ndens))
    return set_error(LTJK_EINVAL, "cd_jk: bad sizes (naux %d, ndens %d, rank %d, u_count %d)", naux, ndens,
                     rank, u_count);
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int N = ctx->nao;
  const size_t NN = (size_t)N * N, per = (size_t)N * rank;
  const size_t u_stride = u_count == 1 ? 0 : per;
  const dim3 thr(16, 16);
  int rc;
  double *gamma;
  if (ctx->opts.precision == LTJK_FP64_NATIVE) {
    // IEEE FP64: per density BU = B U, BV = B V, gamma, and K = sum_Q BU BV^T
    const size_t need = (2 * (size_t)naux * per + (size_t)naux * ndens) * sizeof(double);
    if ((rc = ctx->ensure_scratch(need, st))) return rc;
    double *BU = ctx->scratch.as<double>(), *BV = BU + (size_t)naux * per;
    gamma = BV + (size_t)naux * per;
    const long long M = (long long)naux * N;  // B viewed as [naux*N][N]
    const dim3 gbu((unsigned)((M + 15) / 16), (unsigned)((rank + 15) / 16));
    const int tiles = ((N + 15) / 16) * ((N + 15) / 16);
    const int qsplit = std::max(1, std::min(naux, num_sms() * 8 / std::max(1, tiles) + 1));
    const int qchunk = (naux + qsplit - 1) / qsplit;
    for (int q = 0; q < ndens; ++q) {
      const double *Uq = U + (size_t)q * u_stride, *Vq = V + (size_t)q * per;
      if (q == 0 || u_stride) {
        cd_gemm<false><<<gbu, thr, 0, st>>>(B, Uq, BU, M, rank, N, N, rank, rank);
        g_launches += 1;
      }
      cd_gemm<false><<<gbu, thr, 0, st>>>(B, Vq, BV, M, rank, N, N, rank, rank);
      cd_gamma<<<std::min(naux, num_sms() * 8), 256, 0, st>>>(BU, Vq, naux, per, gamma + (size_t)q * naux);
      g_launches += 2;
      if (K) {
        double *Kq = K + (size_t)q * NN;
        CUDA_TRY(cudaMemsetAsync(Kq, 0, NN * sizeof(double), st));
        cd_k_contract<<<dim3((N + 15) / 16, (N + 15) / 16, (naux + qchunk - 1) / qchunk), thr, 0, st>>>(
            BU, BV, naux, N, rank, qchunk, Kq);
        g_launches += 1;
      }
    }
  } else {
    // Double-float GEMMs on the FP32 pipe: B U and B V_q stored as [mu][(Q, m)]
    // so that each K_q is one product with the contracted index (Q, m) contiguous.
    const size_t blk = (size_t)naux * per;  // one [N][naux][rank] block
    int chunk = std::max(1, std::min(ndens, (int)((size_t(2) << 30) / (blk * sizeof(double)))));
    const size_t nblk_u = u_stride ? (size_t)chunk : 1;
    const size_t need = (blk * (nblk_u + chunk) + per * (nblk_u + chunk) + (size_t)naux * ndens) * sizeof(double);
    if ((rc = ctx->ensure_scratch(need, st))) return rc;
    double *BU = ctx->scratch.as<double>(), *BV = BU + blk * nblk_u, *Vt = BV + blk * chunk,
           *Ut = Vt + per * chunk;
    gamma = Ut + per * nblk_u;
    const PermShape ps{N, naux, rank};
    const long long M = (long long)naux * N;
    const long long kd = (long long)naux * rank;
    const int ktiles = ((N + 63) / 64) * ((N + 63) / 64);
    const int zsplit = (int)std::max<long long>(1, std::min<long long>((kd + 15) / 16, (num_sms() * 3 + ktiles - 1) / ktiles));
    const long long kchunk = ((kd + zsplit - 1) / zsplit + 15) / 16 * 16;
    const int gz = (int)((kd + kchunk - 1) / kchunk);
    for (int q0 = 0; q0 < ndens; q0 += chunk) {
      const int nc = std::min(chunk, ndens - q0);
      // left factors: shared U once, else one per density of the chunk
      if (q0 == 0 || u_stride) {
        const int nu = u_stride ? nc : 1;
        const double *Uq = U + (size_t)q0 * u_stride;
        cd_transpose_factors<<<(int)std::min<size_t>((per * nu + 255) / 256, num_sms() * 16), 256, 0, st>>>(
            Uq, nu, N, rank, Ut);
        cd_gemm_nt_df<kEpiPerm><<<dim3((unsigned)((M + 63) / 64), (unsigned)((nu * rank + 63) / 64), 1), 256, 0,
                                  st>>>(B, N, Ut, N, BU, 0, M, nu * rank, N, N, ps);
        g_launches += 2;
      }
      cd_transpose_factors<<<(int)std::min<size_t>((per * nc + 255) / 256, num_sms() * 16), 256, 0, st>>>(
          V + (size_t)q0 * per, nc, N, rank, Vt);
      cd_gemm_nt_df<kEpiPerm><<<dim3((unsigned)((M + 63) / 64), (unsigned)((nc * rank + 63) / 64), 1), 256, 0,
                                st>>>(B, N, Vt, N, BV, 0, M, nc * rank, N, N, ps);
      cd_gamma_perm<<<(int)std::min<long long>(((long long)nc * naux * 32 + 255) / 256, num_sms() * 32), 256, 0, st>>>(
          BU, u_stride ? blk : 0, V + (size_t)q0 * per, nc, naux, N, rank, gamma + (size_t)q0 * naux);
      g_launches += 3;
      if (K && !u_stride) {
        // one product for the whole chunk: K[mu][(j, nu)] = sum BU[mu][.] BV_j[nu][.],
        // the densities stacked along the columns (BV is [j][nu][(Q, m)])
        CUDA_TRY(cudaMemsetAsync(K + (size_t)q0 * NN, 0, (size_t)nc * NN * sizeof(double), st));
        const int ctiles = (nc * N + 63) / 64, rtiles = (N + 63) / 64;
        const int zk = (int)std::max<long long>(1, std::min<long long>((kd + 15) / 16,
                                                                        (num_sms() * 3 + rtiles * ctiles - 1) / (rtiles * ctiles)));
        const long long kchunk_c = ((kd + zk - 1) / zk + 15) / 16 * 16;
        const int gzc = (int)((kd + kchunk_c - 1) / kchunk_c);
        cd_gemm_nt_df<kEpiAtomicK><<<dim3(rtiles, ctiles, gzc), 256, 0, st>>>(
            BU, (int)kd, BV, (int)kd, K + (size_t)q0 * NN, N, N, nc * N, kd, kchunk_c, ps);
        g_launches += 1;
      } else if (K) {
        for (int j = 0; j < nc; ++j) {
          const int q = q0 + j;
          double *Kq = K + (size_t)q * NN;
          const double *BUq = BU + (size_t)j * blk;
          CUDA_TRY(cudaMemsetAsync(Kq, 0, NN * sizeof(double), st));
          cd_gemm_nt_df<kEpiAtomic><<<dim3((N + 63) / 64, (N + 63) / 64, gz), 256, 0, st>>>(
              BUq, (int)kd, BV + (size_t)j * blk, (int)kd, Kq, N, N, N, kd, kchunk, ps);
          g_launches += 1;
        }
      }
    }
  }
  if (J) {
    // J[q] = sum_Q gamma[q][Q] B[Q]   ([ndens][naux] x [naux][N*N]), FP64, in
    // column chunks so that the column tiles stay within grid y's 65535
    const size_t cchunk = (size_t)65535 * 16;
    for (size_t c0 = 0; c0 < NN; c0 += cchunk) {
      const int nc = (int)std::min(cchunk, NN - c0);
      const dim3 gj((unsigned)((ndens + 15) / 16), (unsigned)((nc + 15) / 16));
      cd_gemm<false><<<gj, thr, 0, st>>>(gamma, B + c0, J + c0, ndens, nc, naux, naux, (int)NN, (int)NN);
      g_launches += 1;
    }
  }
  CUDA_TRY(cudaGetLastError());
  return LTJK_OK;
}

}  // extern "C"
