// metrics.cu -- the two clustering scores of the paper's Section 5 on the
// device: the adjusted Rand index (Hubert & Arabie 1985) and the adjusted
// mutual information (Vinh, Epps & Bailey 2010).  Both start from the same
// contingency counts: an open-addressing set of (label a, label b) pairs with
// a count per pair, and a count per label on either side.
#include <cmath>
#include <cstring>

#include "api_common.cuh"

namespace sng {

// ------------------------------------------------------ contingency counts

// Labels are in [-1, n) and indexed by label + 1.  keys start all ones.
__global__ void contingency_kernel(const int32_t *a, const int32_t *b, int64_t n,
                                   unsigned long long *keys, unsigned long long *cnt,
                                   uint64_t cap_mask, unsigned long long *ca,
                                   unsigned long long *cb, unsigned long long *counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(counters + kCntStatus);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t la = (int64_t)a[i] + 1, lb = (int64_t)b[i] + 1;
    if (la < 0 || la > n || lb < 0 || lb > n) {
      atomicOr(status, kErrIndex);
      continue;
    }
    atomicAdd(ca + la, 1ull);
    atomicAdd(cb + lb, 1ull);
    const unsigned long long key = ((unsigned long long)la << 32) | (unsigned long long)lb;
    uint64_t h = mix64(key) & cap_mask;
    bool done = false;
    for (uint64_t probe = 0; probe <= cap_mask; ++probe) {
      const unsigned long long old = atomicCAS(keys + h, ~0ull, key);
      if (old == ~0ull || old == key) {
        atomicAdd(cnt + h, 1ull);
        done = true;
        break;
      }
      h = (h + 1) & cap_mask;
    }
    if (!done) atomicOr(status, kErrIndex);
  }
}

struct Contingency {
  uint64_t cap = 0;
  unsigned long long *keys = nullptr, *cnt = nullptr, *ca = nullptr, *cb = nullptr;
  unsigned long long *counters = nullptr;
};

static sng_status build_contingency(const int32_t *a, const int32_t *b, int64_t n, Scratch &s,
                                    Contingency *c) {
  cudaStream_t st = s.stream;
  c->cap = 1;
  while (c->cap < (uint64_t)(2 * n)) c->cap <<= 1;
  sng_status rc;
  if ((rc = s.alloc((void **)&c->keys, c->cap * 8, "label-pair keys")) ||
      (rc = s.alloc((void **)&c->cnt, c->cap * 8, "label-pair counts")) ||
      (rc = s.alloc((void **)&c->ca, (size_t)(n + 1) * 8, "label counts a")) ||
      (rc = s.alloc((void **)&c->cb, (size_t)(n + 1) * 8, "label counts b")) ||
      (rc = s.alloc((void **)&c->counters, kCntSlots * 8, "metric sums")))
    return rc;
  cudaMemsetAsync(c->keys, 0xff, c->cap * 8, st);
  cudaMemsetAsync(c->cnt, 0, c->cap * 8, st);
  cudaMemsetAsync(c->ca, 0, (size_t)(n + 1) * 8, st);
  cudaMemsetAsync(c->cb, 0, (size_t)(n + 1) * 8, st);
  cudaMemsetAsync(c->counters, 0, kCntSlots * 8, st);
  contingency_kernel<<<device_sms() * 8, 256, 0, st>>>(a, b, n, c->keys, c->cnt, c->cap - 1,
                                                       c->ca, c->cb, c->counters);
  note_launch();
  return SNG_OK;
}

// ------------------------------------------------------------------ ARI

// sum over entries of c*(c-1)/2
__global__ void pairs_kernel(const unsigned long long *cnt, int64_t len,
                             unsigned long long *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
    const unsigned long long c = cnt[i];
    s += c * (c - (c ? 1ull : 0ull)) / 2ull;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFullMask, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// ------------------------------------------------------------------ AMI

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

// MI = sum over non-empty cells of (c/n) log(n c / (a b)).
__global__ void mi_kernel(const unsigned long long *keys, const unsigned long long *cnt,
                          int64_t cap, const unsigned long long *ca,
                          const unsigned long long *cb, double n, double *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double s = 0.0;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < cap; h += stride) {
    const unsigned long long c = cnt[h];
    if (!c) continue;
    const unsigned long long key = keys[h];
    const double a = (double)ca[key >> 32], b = (double)cb[key & 0xffffffffull];
    const double cd = (double)c;
    s += cd / n * log(n * cd / (a * b));
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// Non-empty entries of cnt[0, len) appended to (idx_out[k], val_out[k])
// (either may be NULL); *len_out counts them.  Order is irrelevant: every
// consumer only sums over the list.
__global__ void compact_kernel(const unsigned long long *cnt, int64_t len, int64_t *idx_out,
                               unsigned long long *val_out, unsigned long long *len_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  // whole warps walk the range together so the ballot below sees every lane
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < len;
       base += stride) {
    const int64_t i = base + lane;
    const unsigned long long c = i < len ? cnt[i] : 0ull;
    const uint32_t mask = __ballot_sync(kFullMask, c != 0);
    if (!mask) continue;
    unsigned long long first = 0;
    if (lane == 0) first = atomicAdd(len_out, (unsigned long long)__popc(mask));
    first = __shfl_sync(kFullMask, first, 0);
    if (c) {
      const int64_t k = (int64_t)first + __popc(mask & ((1u << lane) - 1u));
      if (idx_out) idx_out[k] = i;
      if (val_out) val_out[k] = c;
    }
  }
}

// H = -sum (s/n) log(s/n) over a list of cluster sizes.
__global__ void entropy_kernel(const unsigned long long *sizes, int64_t len, double n,
                               double *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride) {
    const double p = (double)sizes[k] / n;
    s -= p * log(p);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// Histogram of cluster sizes: hist[size] += 1.
__global__ void size_hist_kernel(const unsigned long long *sizes, int64_t len,
                                 unsigned long long *hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride)
    atomicAdd(hist + sizes[k], 1ull);
}

// Expected MI contribution of one pair of cluster sizes (a, b) among n
// points: sum over cell counts k >= 1 of (k/n) log(n k / (a b)) P(k), P the
// hypergeometric law of the overlap of a random a-subset with a fixed
// b-subset.  P is unimodal with its mode at floor((a+1)(b+1)/(n+2)); P(mode)
// comes from log-gamma values (at least 1/(min(a,b)+1), so it does not
// underflow) and the other terms from the ratios
//   P(k+1)/P(k) = (a-k)(b-k) / ((k+1)(n-a-b+k+1))
// walking outwards.  P is log-concave, so along each walk the ratios only
// shrink: once a ratio r is below 1 the terms still ahead sum to at most
// P r / (1 - r) times the largest weight |(k/n) log(n k / (a b))| on the
// support, and the walk stops when that bound falls below 2^-60 of the sum
// so far (or P underflows, or the support ends).
__device__ double emi_pair(double a, double b, double n, double lg_n1) {
  const double lo = fmax(1.0, a + b - n), hi = fmin(a, b);
  if (lo > hi) return 0.0;
  double mode = floor((a + 1.0) * (b + 1.0) / (n + 2.0));
  mode = fmin(fmax(mode, lo), hi);
  const double logp = lgamma(a + 1.0) + lgamma(b + 1.0) + lgamma(n - a + 1.0) +
                      lgamma(n - b + 1.0) - lg_n1 - lgamma(mode + 1.0) -
                      lgamma(a - mode + 1.0) - lgamma(b - mode + 1.0) -
                      lgamma(n - a - b + mode + 1.0);
  const double p0 = exp(logp);
  const double ab = a * b;
  // |weight| <= (hi/n) max(|log(n lo/(a b))|, |log(n hi/(a b))|): the log is
  // monotone in k and k/n <= hi/n
  const double wmax = hi / n * fmax(fabs(log(n * lo / ab)), fabs(log(n * hi / ab)));
  const double tiny = 0x1p-60;
  double sum = mode / n * log(n * mode / ab) * p0;
  double p = p0;
  for (double k = mode; k < hi;) {
    const double r = ((a - k) * (b - k)) / ((k + 1.0) * (n - a - b + k + 1.0));
    p *= r;
    k += 1.0;
    if (p == 0.0) break;
    sum += k / n * log(n * k / ab) * p;
    if (r < 1.0 && wmax * p * r / (1.0 - r) <= tiny * fabs(sum)) break;
  }
  p = p0;
  for (double k = mode; k > lo;) {
    const double r = (k * (n - a - b + k)) / ((a - k + 1.0) * (b - k + 1.0));
    p *= r;
    k -= 1.0;
    if (p == 0.0) break;
    sum += k / n * log(n * k / ab) * p;
    if (r < 1.0 && wmax * p * r / (1.0 - r) <= tiny * fabs(sum)) break;
  }
  return sum;
}

// E[MI] = sum over distinct size pairs of mult_a * mult_b * emi_pair.
__global__ void emi_kernel(const int64_t *size_a, const unsigned long long *mult_a, int64_t ra,
                           const int64_t *size_b, const unsigned long long *mult_b, int64_t rb,
                           double n, double lg_n1, double *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t pairs = ra * rb;
  double s = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < pairs; t += stride) {
    const int64_t u = t / rb, v = t - u * rb;
    const double w = (double)mult_a[u] * (double)mult_b[v];
    s += w * emi_pair((double)size_a[u], (double)size_b[v], n, lg_n1);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

static int grid_for(int64_t work, int sms) {
  int64_t b = (work + 255) / 256;
  if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace sng

using namespace sng;

extern "C" {

sng_status sng_ari(const int32_t *a, const int32_t *b, int64_t n, double *ari, void *stream) {
  NvtxRange nvtx_range("sng_ari");
  if (!a || !b || !ari) return fail(SNG_EINVAL, "NULL argument");
  if (n < 0 || n > 0x7fffffffLL) return fail(SNG_EINVAL, "n out of range");
  if (n < 2) {
    *ari = 1.0;
    return SNG_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  Contingency c;
  sng_status rc;
  if ((rc = build_contingency(a, b, n, s, &c))) return rc;
  const int sms = device_sms();
  pairs_kernel<<<sms * 8, 256, 0, st>>>(c.cnt, (int64_t)c.cap, c.counters + 0);
  pairs_kernel<<<sms * 8, 256, 0, st>>>(c.ca, n + 1, c.counters + 1);
  pairs_kernel<<<sms * 8, 256, 0, st>>>(c.cb, n + 1, c.counters + 2);
  note_launch(3);
  unsigned long long h[kCntSlots];
  cudaError_t e = cudaMemcpyAsync(h, c.counters, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ari");
  if ((uint32_t)h[kCntStatus]) return fail(SNG_EINVAL, "labels outside [-1, n)");
  const double index = (double)h[0], sa = (double)h[1], sb = (double)h[2];
  const double total = (double)n * (double)(n - 1) / 2.0;
  const double expected = sa * sb / total;
  const double maxi = 0.5 * (sa + sb);
  *ari = (maxi == expected) ? 1.0 : (index - expected) / (maxi - expected);
  return SNG_OK;
}

sng_status sng_ami(const int32_t *a, const int32_t *b, int64_t n, int32_t average,
                   sng_mi_terms *out, void *stream) {
  NvtxRange nvtx_range("sng_ami");
  if (!a || !b || !out) return fail(SNG_EINVAL, "NULL argument");
  if (n < 0 || n > 0x7fffffffLL) return fail(SNG_EINVAL, "n out of range");
  if (average < SNG_AMI_MIN || average > SNG_AMI_MAX) return fail(SNG_EINVAL, "unknown average");
  std::memset(out, 0, sizeof(*out));
  if (n < 2) {
    out->ami = 1.0;
    out->clusters_a = out->clusters_b = n;
    return SNG_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  Contingency c;
  sng_status rc;
  if ((rc = build_contingency(a, b, n, s, &c))) return rc;
  const int sms = device_sms();
  const double nd = (double)n;
  // counters slots 0-3 hold FP64 sums: MI, H_a, H_b, E[MI]; 4-7 list lengths
  double *sums = reinterpret_cast<double *>(c.counters);
  unsigned long long *lens = c.counters + 4;
  mi_kernel<<<grid_for((int64_t)c.cap, sms), 256, 0, st>>>(c.keys, c.cnt, (int64_t)c.cap, c.ca,
                                                           c.cb, nd, sums + 0);
  // cluster sizes of either side, then their entropies
  unsigned long long *size_a, *size_b, *mult_a, *mult_b;
  int64_t *dsize_a, *dsize_b;
  if ((rc = s.alloc((void **)&size_a, (size_t)(n + 1) * 8, "cluster sizes a")) ||
      (rc = s.alloc((void **)&size_b, (size_t)(n + 1) * 8, "cluster sizes b")))
    return rc;
  compact_kernel<<<grid_for(n + 1, sms), 256, 0, st>>>(c.ca, n + 1, nullptr, size_a, lens + 0);
  compact_kernel<<<grid_for(n + 1, sms), 256, 0, st>>>(c.cb, n + 1, nullptr, size_b, lens + 1);
  unsigned long long h[kCntSlots];
  cudaError_t e = cudaMemcpyAsync(h, c.counters, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ami");
  if ((uint32_t)h[kCntStatus]) return fail(SNG_EINVAL, "labels outside [-1, n)");
  const int64_t ra = (int64_t)h[4], rb = (int64_t)h[5];
  entropy_kernel<<<grid_for(ra, sms), 256, 0, st>>>(size_a, ra, nd, sums + 1);
  entropy_kernel<<<grid_for(rb, sms), 256, 0, st>>>(size_b, rb, nd, sums + 2);
  // distinct sizes with multiplicities: E[MI] depends on the sizes only, so
  // pairs of equal sizes are evaluated once (at most ~sqrt(2n) distinct
  // sizes per side, however many clusters there are)
  cudaMemsetAsync(c.ca, 0, (size_t)(n + 1) * 8, st);
  cudaMemsetAsync(c.cb, 0, (size_t)(n + 1) * 8, st);
  size_hist_kernel<<<grid_for(ra, sms), 256, 0, st>>>(size_a, ra, c.ca);
  size_hist_kernel<<<grid_for(rb, sms), 256, 0, st>>>(size_b, rb, c.cb);
  if ((rc = s.alloc((void **)&dsize_a, (size_t)ra * 8, "distinct sizes a")) ||
      (rc = s.alloc((void **)&dsize_b, (size_t)rb * 8, "distinct sizes b")) ||
      (rc = s.alloc((void **)&mult_a, (size_t)ra * 8, "size multiplicities a")) ||
      (rc = s.alloc((void **)&mult_b, (size_t)rb * 8, "size multiplicities b")))
    return rc;
  compact_kernel<<<grid_for(n + 1, sms), 256, 0, st>>>(c.ca, n + 1, dsize_a, mult_a, lens + 2);
  compact_kernel<<<grid_for(n + 1, sms), 256, 0, st>>>(c.cb, n + 1, dsize_b, mult_b, lens + 3);
  note_launch(9);
  e = cudaMemcpyAsync(h, c.counters, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ami");
  const int64_t da = (int64_t)h[6], db = (int64_t)h[7];
  emi_kernel<<<grid_for(da * db, sms), 256, 0, st>>>(dsize_a, mult_a, da, dsize_b, mult_b, db,
                                                     nd, std::lgamma(nd + 1.0), sums + 3);
  note_launch();
  e = cudaMemcpyAsync(h, c.counters, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ami");
  double v[4];
  std::memcpy(v, h, sizeof(v));
  out->mi = v[0];
  out->h_a = v[1];
  out->h_b = v[2];
  out->emi = v[3];
  out->clusters_a = ra;
  out->clusters_b = rb;
  if ((ra == 1 && rb == 1) || (ra == n && rb == n)) {
    out->ami = 1.0;
    return SNG_OK;
  }
  double norm;
  switch (average) {
    case SNG_AMI_MIN: norm = std::fmin(v[1], v[2]); break;
    case SNG_AMI_GEOMETRIC: norm = std::sqrt(v[1] * v[2]); break;
    case SNG_AMI_ARITHMETIC: norm = 0.5 * (v[1] + v[2]); break;
    default: norm = std::fmax(v[1], v[2]); break;
  }
  const double den = norm - v[3];
  out->ami = den <= 0.0 ? 0.0 : (v[0] - v[3]) / den;
  return SNG_OK;
}

}  // extern "C"
