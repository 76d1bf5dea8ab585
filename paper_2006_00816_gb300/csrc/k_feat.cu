// k_feat.cu -- energy, block normalisation, truncation and the 31 features
// (Section 4.1.1: normalisation and feature computation; Section 5.1,
// energy and feature kernels, fused here into one pass).
//
// Energy of a cell: E = sum_{n<9} (h_n + h_{n+9})^2, zero outside the grid.
// The four 2x2-cell blocks containing cell (i, j) extend towards (dx, dy) =
// (-1,-1), (+1,-1), (-1,+1), (+1,+1); S_k is the sum of their energies and
// N_k = 1/sqrt(S_k + eps).  Features, truncated at tau:
//   f[o]      = 1/2    sum_k min(h_o N_k, tau)            o < 18 (signed)
//   f[18+o]   = 1/2    sum_k min((h_o + h_{o+9}) N_k, tau) o < 9 (unsigned)
//   f[27+k]   = 0.2357 sum_o min(h_o N_k, tau)            k < 4 (energy)
// Output: the internal layout [4 chunks][cy][cx][8 channels] (channel 31 is
// a zero pad so that the correlation streams 8-channel float4 pairs), and
// optionally the user layout [cy][cx][31].
#include "hog_internal.cuh"

namespace hogk {

namespace {
constexpr int HX = FEAT_TX + 2;   // 34 halo columns
constexpr int HY = FEAT_TY + 2;   // 10 halo rows
constexpr int CS = NBIN + 1;      // padded cell stride in shared memory
constexpr int NT = FEAT_TX * FEAT_TY;
}  // namespace

__global__ void __launch_bounds__(NT) feat_kernel(const LevelDesc *__restrict__ descs,
                                                  const Job *__restrict__ jobs, float eps,
                                                  float tau) {
    __shared__ float hS[HY * HX * CS];
    __shared__ float eS[HY * HX];
    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int ntx = (d.cx + FEAT_TX - 1) / FEAT_TX;
    const int j0 = (jb.tile % ntx) * FEAT_TX, i0 = (jb.tile / ntx) * FEAT_TY;
    const int t = threadIdx.x;

    // halo cells [i0-1, i0+FEAT_TY] x [j0-1, j0+FEAT_TX], zero outside the grid
    for (int k = t; k < HY * HX * NBIN; k += NT) {
        const int r = k / (HX * NBIN);
        const int rem = k - r * HX * NBIN;
        const int c = rem / NBIN, b = rem - c * NBIN;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        float v = 0.0f;
        if (i >= 0 && i < d.cy && j >= 0 && j < d.cx)
            v = __ldg(d.hist + ((size_t)i * d.cx + j) * NBIN + b);
        hS[(r * HX + c) * CS + b] = v;
    }
    __syncthreads();
    for (int k = t; k < HY * HX; k += NT) {
        const float *h = hS + k * CS;
        float e = 0.0f;
#pragma unroll
        for (int n = 0; n < 9; n++) {
            const float s = h[n] + h[n + 9];
            e += s * s;
        }
        eS[k] = e;
    }
    __syncthreads();

    const int ti = t / FEAT_TX, tj = t - ti * FEAT_TX;
    const int i = i0 + ti, j = j0 + tj;
    if (i >= d.cy || j >= d.cx) return;
    const int r = ti + 1, c = tj + 1;
    const float *h = hS + (r * HX + c) * CS;
    float hv[NBIN];
#pragma unroll
    for (int b = 0; b < NBIN; b++) hv[b] = h[b];

    const float e00 = eS[r * HX + c];
    const float S0 = e00 + eS[r * HX + c - 1] + eS[(r - 1) * HX + c] + eS[(r - 1) * HX + c - 1];
    const float S1 = e00 + eS[r * HX + c + 1] + eS[(r - 1) * HX + c] + eS[(r - 1) * HX + c + 1];
    const float S2 = e00 + eS[r * HX + c - 1] + eS[(r + 1) * HX + c] + eS[(r + 1) * HX + c - 1];
    const float S3 = e00 + eS[r * HX + c + 1] + eS[(r + 1) * HX + c] + eS[(r + 1) * HX + c + 1];
    const float N0 = 1.0f / sqrtf(S0 + eps), N1 = 1.0f / sqrtf(S1 + eps);
    const float N2 = 1.0f / sqrtf(S2 + eps), N3 = 1.0f / sqrtf(S3 + eps);

    float f[32];
    float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
#pragma unroll
    for (int o = 0; o < NBIN; o++) {
        const float a0 = fminf(hv[o] * N0, tau), a1 = fminf(hv[o] * N1, tau);
        const float a2 = fminf(hv[o] * N2, tau), a3 = fminf(hv[o] * N3, tau);
        f[o] = 0.5f * (((a0 + a1) + a2) + a3);
        t0 += a0; t1 += a1; t2 += a2; t3 += a3;
    }
#pragma unroll
    for (int o = 0; o < 9; o++) {
        const float s = hv[o] + hv[o + 9];
        const float a0 = fminf(s * N0, tau), a1 = fminf(s * N1, tau);
        const float a2 = fminf(s * N2, tau), a3 = fminf(s * N3, tau);
        f[NBIN + o] = 0.5f * (((a0 + a1) + a2) + a3);
    }
    f[27] = 0.2357f * t0;
    f[28] = 0.2357f * t1;
    f[29] = 0.2357f * t2;
    f[30] = 0.2357f * t3;
    f[31] = 0.0f;

    const size_t plane = (size_t)d.cy * d.cx * CHUNK;
    const size_t cell = (size_t)i * d.cx + j;
#pragma unroll
    for (int ch = 0; ch < NCHUNK; ch++) {
        float4 *dst = reinterpret_cast<float4 *>(d.feat + ch * plane + cell * CHUNK);
        dst[0] = make_float4(f[8 * ch + 0], f[8 * ch + 1], f[8 * ch + 2], f[8 * ch + 3]);
        dst[1] = make_float4(f[8 * ch + 4], f[8 * ch + 5], f[8 * ch + 6], f[8 * ch + 7]);
    }
    if (d.feat_user) {
        float *u = d.feat_user + cell * NFEAT;
#pragma unroll
        for (int o = 0; o < NFEAT; o++) u[o] = f[o];
    }
}

cudaError_t launch_feat(const LevelDesc *descs, const Job *jobs, int njobs, float eps,
                        float tau, cudaStream_t stream) {
    if (njobs <= 0) return cudaSuccess;
    feat_kernel<<<njobs, NT, 0, stream>>>(descs, jobs, eps, tau);
    return cudaGetLastError();
}

}  // namespace hogk
