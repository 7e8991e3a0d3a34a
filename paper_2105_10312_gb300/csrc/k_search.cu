// k_search.cu — exact optimum over every SM split and task-to-partition map
// (the exhaustive yardstick for the heuristic of §5).
//
// The explicit space is every composition of M/g into k in [kmin, kmax]
// parts times every map of the n tasks to the k parts.  Because the test is
// monotone in m (§4.1) and in the task set, that space reduces exactly to
// set partitions of the tasks: a set partition with b blocks is realisable
// iff b <= kmax, every block has a minimum size minm(block) <= M, and
// sum minm + max(0, kmin - b) g <= M (empty parts still take g SMs).  So one
// CTA per task set
//   phase A: computes minm(S) and the inflated workload W(S) of every
//            non-empty subset S (one thread per subset, serial test);
//   phase B: sweeps every restricted-growth string (RGS) with at most kmax
//            blocks (threads take contiguous rank ranges), keeps the
//            smallest key (W, sum minm, RGS), and reduces it over the CTA.
#include <cuda_runtime.h>

#include "gpa_device.cuh"
#include "gpa_internal.h"

namespace gpa {

namespace {

constexpr int kSN = GPA_SEARCH_NMAX;  // tasks per set
constexpr int kSK = GPA_SEARCH_KMAX;  // blocks per set partition
constexpr int kSThreads = 256;

struct SearchHead {
  unsigned int T[kSN], D[kSN], mT[kSN], sh[kSN];
  unsigned long long A[kSN], B[kSN];
  unsigned int u[kSN];
  unsigned int memmask;        // rows of memory tasks
  unsigned int rowbit[kSN];    // original task -> bit of its DM row
  unsigned int singleton[kSN]; // Lemma 2 size of each row
  unsigned long long cnt[kSN + 1][kSK + 2];  // RGS completion counts
  unsigned long long bestK1[kSThreads / 32];
  unsigned long long bestK2[kSThreads / 32];
  int n;
  long long set;
};

// Serial per-partition test (one thread): rows of S in priority order at m.
__device__ bool serial_rta(const SearchHead& h, unsigned int S, unsigned int m, unsigned int kc, unsigned int km,
                           const MagicDiv& md) {
  const int nm = __popc(S & h.memmask), ns = __popc(S);
  const unsigned int kmem = nm >= 2 ? km : 1000u, kcmp = (ns - nm) >= 2 ? kc : 1000u;
  unsigned int C[kSN];
  unsigned long long prefix = 0;
  for (unsigned int rest = S; rest; rest &= rest - 1u) {
    const int i = __ffs(rest) - 1;
    const unsigned int Ci = wcet(h.A[i], h.B[i], ((h.memmask >> i) & 1u) ? kmem : kcmp, m, md);
    C[i] = Ci;
    unsigned long long R = prefix + Ci;
    prefix = R;
    const unsigned int Di = h.D[i];
    const unsigned int hp = S & ((1u << i) - 1u);
    int iter = 0;
    for (;;) {
      if (R > Di) return false;
      const unsigned long long cap = (unsigned long long)Di + 1ull;
      unsigned long long next = Ci;
      for (unsigned int r2 = hp; r2; r2 &= r2 - 1u) {
        const int j = __ffs(r2) - 1;
        const unsigned long long t = (unsigned long long)ceil_div_T((unsigned int)R, h.mT[j], h.sh[j]) * C[j];
        next += t < cap ? t : cap;
      }
      if (next == R) break;
      R = next;
      if (++iter > kIterCap) return false;
    }
  }
  return true;
}

// smallest multiple of g in [g, M] at which S passes (0 if none): binary
// search between the largest singleton size of S and M.
__device__ unsigned int serial_minm(const SearchHead& h, unsigned int S, const DevModel& md,
                                    const MagicDiv* __restrict__ mdiv) {
  unsigned int lo = md.g;
  for (unsigned int r = S; r; r &= r - 1u) {
    const unsigned int z = h.singleton[__ffs(r) - 1];
    if (z == 0u) return 0u;
    lo = max(lo, z);
  }
  const unsigned int g = md.g, M = md.M;
  if (!serial_rta(h, S, M, md.kc, md.km, mdiv[M])) return 0u;
  unsigned int a = lo / g, b = M / g;
  while (a < b) {
    const unsigned int mid = a + (b - a) / 2u;
    if (serial_rta(h, S, mid * g, md.kc, md.km, mdiv[mid * g])) b = mid;
    else a = mid + 1u;
  }
  return a * g;
}

__device__ __forceinline__ bool key_less(unsigned long long a1, unsigned long long a2, unsigned long long b1,
                                         unsigned long long b2) {
  return a1 < b1 || (a1 == b1 && a2 < b2);
}

__global__ void __launch_bounds__(kSThreads) search_sets(DevSets S, DevModel md, int kmin, int kmax, BestOut out,
                                                         unsigned int* err, const MagicDiv* __restrict__ mdiv,
                                                         unsigned long long* ticket, int nsub_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SearchHead& h = *reinterpret_cast<SearchHead*>(smem_raw);
  unsigned long long* Wsub = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(SearchHead));
  unsigned short* msub = reinterpret_cast<unsigned short*>(Wsub + nsub_max);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long kNoKey = ~0ull;

  for (;;) {
    __syncthreads();
    if (tid == 0) h.set = (long long)atomicAdd(ticket, 1ull);
    __syncthreads();
    const long long s = h.set;
    if (s >= S.nsets) break;
    const long long o = S.set_off[s];
    const long long nl = S.set_off[s + 1] - o;
    // ---- stage (warp 0): validate, DM order, Lemma 2 sizes
    bool bad = nl < 0 || nl > kSN || (1ll << (nl < 0 ? 0 : nl)) > nsub_max;
    const int n = bad ? 0 : (int)nl;
    if (warp == 0) {
      bool ok = !bad;
      long long Tt = 0, Dt = 0, At = 0, Bt = 0, ut = 0;
      unsigned int yt = 0;
      if (ok && lane < n) {
        Tt = S.T[o + lane];
        Dt = S.D[o + lane];
        At = S.A[o + lane];
        Bt = S.B[o + lane];
        ut = S.u[o + lane];
        yt = S.type[o + lane];
        ok = task_valid(Tt, Dt, At, Bt, ut, yt);
      }
      ok = __all_sync(kFull, ok);
      // deadline-monotonic rank by all-pairs compare through shuffles
      int r = 0;
      const unsigned long long key = ((unsigned long long)Dt << 31) | (unsigned long long)Tt;
      for (int j = 0; j < kSN; j++) {
        const unsigned long long kj = __shfl_sync(kFull, key, j);
        if (ok && lane < n && j < n) r += (kj < key) || (kj == key && j < lane);
      }
      if (ok && lane < n) {
        h.T[r] = (unsigned int)Tt;
        h.D[r] = (unsigned int)Dt;
        unsigned int mg, sh;
        magic_for_period((unsigned int)Tt, &mg, &sh);
        h.mT[r] = mg;
        h.sh[r] = sh;
        h.A[r] = (unsigned long long)At;
        h.B[r] = (unsigned long long)Bt;
        h.u[r] = (unsigned int)ut;
        h.rowbit[lane] = 1u << r;
        h.singleton[r] = lemma2_size((unsigned long long)At, (unsigned long long)Bt, (unsigned long long)Dt,
                                     (unsigned)md.M, (unsigned)md.g);
      }
      const unsigned int mem = __ballot_sync(kFull, ok && lane < n && yt == 1u);
      // memmask over rows: rebuild from the rank of each memory task
      unsigned int mm = 0u;
      for (int j = 0; j < kSN; j++) {
        const int rj = __shfl_sync(kFull, r, j);
        if ((mem >> j) & 1u) mm |= 1u << rj;
      }
      if (lane == 0) {
        h.memmask = mm;
        h.n = ok ? n : -1;
      }
      // RGS completion counts: cnt[i][j] = ways to label positions i..n-1
      // with j blocks already open and at most kmax blocks in total
      if (lane == 0 && ok) {
        for (int j = 0; j <= kmax + 1; j++) h.cnt[n][j] = 1ull;
        for (int i = n - 1; i >= 0; i--)
          for (int j = 0; j <= kmax; j++) {
            unsigned long long c = (unsigned long long)j * h.cnt[i + 1][j];
            if (j < kmax) c += h.cnt[i + 1][j + 1];
            h.cnt[i][j] = c;
          }
      }
    }
    __syncthreads();
    if (h.n < 0) {
      if (tid == 0) {
        out.feasible[s] = 0;
        out.W[s] = 0;
        out.sum_minm[s] = 0;
        out.n_blocks[s] = 0;
        out.spare[s] = 0;
        atomicOr(err, kErrRange);
      }
      for (int b = tid; b < kmax; b += kSThreads) out.minm_block[s * kmax + b] = 0;
      for (long long t = tid; t < nl && nl > 0; t += kSThreads) out.rgs[o + t] = 255;
      continue;
    }
    if (n == 0) {
      if (tid == 0) {
        const bool f = (long long)kmin * md.g <= md.M;
        out.feasible[s] = f ? 1 : 0;
        out.W[s] = 0;
        out.sum_minm[s] = 0;
        out.n_blocks[s] = 0;
        out.spare[s] = f ? md.M - kmin * md.g : 0;
      }
      for (int b = tid; b < kmax; b += kSThreads) out.minm_block[s * kmax + b] = 0;
      continue;
    }
    // ---- phase A: minm and W of every non-empty subset of rows
    const unsigned int nsub = 1u << n;
    for (unsigned int S2 = tid; S2 < nsub; S2 += kSThreads) {
      if (S2 == 0u) {
        msub[0] = 0;
        Wsub[0] = 0;
        continue;
      }
      msub[S2] = (unsigned short)serial_minm(h, S2, md, mdiv);
      const int nmS = __popc(S2 & h.memmask), ncS = __popc(S2) - nmS;
      unsigned long long Uc = 0, Um = 0;
      for (unsigned int r = S2; r; r &= r - 1u) {
        const int i = __ffs(r) - 1;
        ((h.memmask >> i) & 1u ? Um : Uc) += h.u[i];
      }
      Wsub[S2] = workload_from_sums(Uc, Um, ncS, nmS, md.kc, md.km);
    }
    __syncthreads();
    // ---- phase B: every RGS with <= kmax blocks, contiguous rank ranges
    const unsigned long long total = h.cnt[1][1];
    const unsigned long long per = (total + kSThreads - 1) / kSThreads;
    const unsigned long long r0 = per * tid;
    const unsigned long long r1 = min(total, r0 + per);
    unsigned long long best1 = kNoKey, best2 = kNoKey;
    if (r0 < r1) {
      unsigned char a[kSN];
      // unrank r0
      a[0] = 0;
      unsigned long long rank = r0;
      int used = 1;
      for (int i = 1; i < n; i++) {
        const int top = used < kmax ? used : kmax - 1;
        for (int b = 0; b <= top; b++) {
          const int nu = b + 1 > used ? b + 1 : used;
          const unsigned long long c = h.cnt[i + 1][nu];
          if (rank < c) {
            a[i] = (unsigned char)b;
            used = nu;
            break;
          }
          rank -= c;
        }
      }
      for (unsigned long long r = r0; r < r1; r++) {
        unsigned int mask[kSK];
        int nb = 0;
#pragma unroll
        for (int b = 0; b < kSK; b++) mask[b] = 0u;
        unsigned long long packed = 0ull;
        for (int i = 0; i < n; i++) {
          mask[a[i]] |= h.rowbit[i];
          nb = max(nb, (int)a[i] + 1);
          packed = (packed << 3) | a[i];
        }
        unsigned int sm = 0u;
        unsigned long long W = 0ull;
        bool ok = true;
        for (int b = 0; b < nb; b++) {
          const unsigned int z = msub[mask[b]];
          ok = ok && z != 0u;
          sm += z;
          W += Wsub[mask[b]];
        }
        const int empty = kmin > nb ? kmin - nb : 0;
        if (ok && (long long)sm + (long long)empty * md.g <= md.M) {
          const unsigned long long k1 = (W << 11) | sm;
          if (key_less(k1, packed, best1, best2)) {
            best1 = k1;
            best2 = packed;
          }
        }
        // lexicographic successor: bump the last position that can grow
        if (r + 1 < r1) {
          unsigned char pm[kSN];
          pm[0] = 0;
          for (int i = 1; i < n; i++) pm[i] = max(pm[i - 1], (unsigned char)(a[i - 1]));
          int i = n - 1;
          for (; i >= 1; i--) {
            const int lim = min((int)pm[i] + 1, kmax - 1);
            if (a[i] < lim) break;
          }
          a[i]++;
          for (int j = i + 1; j < n; j++) a[j] = 0;
        }
      }
    }
    // ---- CTA argmin of (k1, k2)
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o1 = __shfl_xor_sync(kFull, best1, off);
      const unsigned long long o2 = __shfl_xor_sync(kFull, best2, off);
      if (key_less(o1, o2, best1, best2)) {
        best1 = o1;
        best2 = o2;
      }
    }
    if (lane == 0) {
      h.bestK1[warp] = best1;
      h.bestK2[warp] = best2;
    }
    __syncthreads();
    if (warp == 0) {
      best1 = lane < kSThreads / 32 ? h.bestK1[lane] : kNoKey;
      best2 = lane < kSThreads / 32 ? h.bestK2[lane] : kNoKey;
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(kFull, best1, off);
        const unsigned long long o2 = __shfl_xor_sync(kFull, best2, off);
        if (key_less(o1, o2, best1, best2)) {
          best1 = o1;
          best2 = o2;
        }
      }
      const bool found = best1 != kNoKey;
      // decode the winning RGS (3 bits per task, task 0 most significant)
      int ai = 0;
      if (lane < n) ai = found ? (int)((best2 >> (3 * (n - 1 - lane))) & 7ull) : 255;
      if (lane < n) out.rgs[o + lane] = (unsigned char)ai;
      // block masks of the winner
      int nb = 0;
      unsigned int bm[kSK];
      for (int b = 0; b < kSK; b++) bm[b] = 0u;
      if (found) {
        for (int i = 0; i < n; i++) {
          const int ab = (int)((best2 >> (3 * (n - 1 - i))) & 7ull);
          bm[ab] |= h.rowbit[i];
          nb = max(nb, ab + 1);
        }
      }
      if (lane < kmax) {
        short z = 0;
        for (int b = 0; b < kSK; b++)
          if (b == lane && b < nb) z = (short)msub[bm[b]];
        out.minm_block[s * kmax + lane] = z;
      }
      if (lane == 0) {
        const unsigned int sm = found ? (unsigned int)(best1 & 2047ull) : 0u;
        const int empty = (found && kmin > nb) ? kmin - nb : 0;
        out.feasible[s] = found ? 1 : 0;
        out.W[s] = found ? (long long)(best1 >> 11) : 0;
        out.sum_minm[s] = (int)sm;
        out.n_blocks[s] = found ? nb : 0;
        out.spare[s] = found ? md.M - (int)sm - empty * md.g : 0;
      }
    }
  }
}

size_t search_smem_bytes(int nsub_max) {
  return sizeof(SearchHead) + (size_t)nsub_max * (sizeof(unsigned long long) + sizeof(unsigned short));
}

}  // namespace

cudaError_t search_kernels_init() {
  return cudaFuncSetAttribute(search_sets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)search_smem_bytes(1 << kSN));
}

cudaError_t launch_search_best(const DevSets& s, const DevModel& md, int kmin, int kmax, const BestOut& out,
                               const AllocQueue& q, const MagicDivHost* mdiv, int sm_count, cudaStream_t st,
                               long long* launches, Prof* prof) {
  int nmax = s.n_max < 0 ? 0 : (s.n_max > kSN ? kSN : s.n_max);
  const int nsub_max = 1 << nmax;
  const size_t smem = search_smem_bytes(nsub_max);
  const int per_sm = smem <= 56 * 1024 ? 4 : (smem <= 110 * 1024 ? 2 : 1);
  long long blocks = (long long)sm_count * per_sm;
  if (blocks > s.nsets) blocks = s.nsets > 0 ? s.nsets : 1;
  unsigned long long* ticket = q.counters + 3;
  unsigned int* err = q.err;
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  search_sets<<<(int)blocks, kSThreads, smem, st>>>(s, md, kmin, kmax, out, err,
                                                     reinterpret_cast<const MagicDiv*>(mdiv), ticket, nsub_max);
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 1;
  return e;
}

}  // namespace gpa
