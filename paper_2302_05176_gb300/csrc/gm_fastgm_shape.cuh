// gm_fastgm_shape.cuh -- the FastGM and plain sketch kernels and their launcher
// for one CTA shape.  gm_sketch.cu includes this file once per shape, inside
// namespace gm, with GM_SHAPE_NS (the shape's namespace) and GM_SHAPE_BLOCK
// (threads per CTA; CTAs per SM = 1024 / GM_SHAPE_BLOCK, 64 registers a thread)
// defined; it has no include guard on purpose.
namespace GM_SHAPE_NS {

constexpr int BLOCK = GM_SHAPE_BLOCK;
constexpr int WARPS = BLOCK / 32;
constexpr int CTAS_PER_SM = 1024 / BLOCK;
constexpr int MAPCAP = GM_MAPCAP;  // displaced positions a light lane can track
// The 512-thread shape compiles the compacted units into its one main kernel
// (taken by a runtime flag); the 1024-thread shape into a second instance
// (MODE_CMP), so that its main kernel keeps the register allocation of the
// short-row path.  Both were measured against the other choice (k = 1024:
// 2.57 against 2.64 ms; k = 4096: 8.60 against 8.68 ms per main kernel).
constexpr bool SHARED_CMP = BLOCK == 512;

struct SmemScalars {
  int pool, hcount, bcount, pcount, c_med, c_heavy, c_pheavy, c_super, c_psuper, unit, last;
  float red_f[WARPS];
  int red_i[WARPS];
  double red_d[WARPS];
  unsigned long long clk[WARPS][NCLK];  // light, 8-lane, 32-lane, dense, barrier wait, setup, finish, total
};
__shared__ SmemScalars sh_scalars;

// Shared memory of the FastGM kernel: registers | light maps, 8-lane hashes or
// warp hashes | ndense dense permutations | per-warp screening buffers.
__host__ __device__ inline size_t fast_area_bytes() {
  const size_t maps = (size_t)MAPCAP * BLOCK * 4, hashes = (size_t)WARPS * HASH_SLOTS * 4;
  const size_t med = (size_t)WARPS * (32 / MED_SW) * MED_SLOTS * 4;
  size_t m = maps > hashes ? maps : hashes;
  return m > med ? m : med;
}
// Per-warp screening buffer of the light path: the survivors of a screening
// batch (32 elements, or 64 when long-row chunks screen two per lane) with their
// 1/v and id (doubles first: 8-byte aligned).
constexpr int WB_N = 32 * GM_SCREEN_PAIR;
constexpr size_t WBUF_BYTES = (size_t)WB_N * (8 + 4 + 4);
__host__ __device__ inline size_t fast_smem_bytes(int k, int ndense) {
  return (size_t)k * sizeof(Reg) + fast_area_bytes() + (size_t)ndense * pi_stride(k) * 2 + (size_t)WARPS * WBUF_BYTES;
}
// The plain kernel: registers | one dense permutation per warp.
__host__ __device__ inline size_t plain_smem_bytes(int k) {
  return (size_t)k * sizeof(Reg) + (size_t)WARPS * pi_stride(k) * 2;
}

// --------------------------------------------------------------------------
// Light path with warp screening.  Elements [lo, lo+n) of the unit; T as bits and
// as an FP32 value (equal as reals).  Elements expected to need more than
// a.light_max arrivals go to the work list, tagged by their expected count.
// --------------------------------------------------------------------------
// The screen of one element of a batch (slot < n): positive weights are counted,
// routed to the work list by their expected arrivals below T, or screened by
// their first arrival; surv = it takes a light lane.
// The id is loaded here when `load_id` (a batch loaded at the screen), else given.
// `slot` is the element's offset from lo; the unit's work list starts at list + lb.
// `passed`: the element already passed this screen at this bound (a compacted
// row's entry), so a light one streams without testing it again.
__device__ __forceinline__ void screen_elem(const SketchArgs& a, int64_t lo, int64_t lb, int n, int slot, double v,
                                            int32_t& idv, bool load_id, float Tf, float kf, SmemScalars& sh,
                                            Counters& cnt, bool& surv, bool passed = false) {
  if (!positive_finite(v)) return;
  ++cnt.elements;
  const float vf = f32_trunc(v);
  const float lam = kf * (1.0f - __expf(-(vf * Tf)));  // expected arrivals <= T (routing only)
  if (lam > a.light_max) {
    // 8-lane work from the front of the unit's list, 32-lane and dense work from
    // its back: each warp phase scans only its own class
    if (lam > a.medium_max)
      a.list[lb + n - 1 - atomicAdd(&sh.bcount, 1)] = (uint32_t)slot | (lam > a.heavy_max ? TAG_SUPER : TAG_HEAVY);
    else
      a.list[lb + atomicAdd(&sh.hcount, 1)] = (uint32_t)slot | TAG_MEDIUM;
  } else if (passed) {
    surv = true;
  } else {
    if (load_id) idv = a.ids[lo + slot];
    const Words wd = philox((uint32_t)idv, 0u, a.key0, a.key1);
    if (screen_out(wd.w1, vf, Tf, kf))
      ++cnt.screened;  // first arrival certainly above T: nothing of it counts
    else
      surv = true;
  }
}

// PF: claim and load each screening batch one batch ahead (long-row chunks, whose
// elements come from HBM); without it a batch is loaded when it is screened
// (short rows, whose weights the row sum has just brought into L2).
// ind (with PF): the unit's n elements are the entries plist[lb, lb + n) of a
// compacted long row, offsets from lo; otherwise elements [lo, lo + n) (lb = lo).
// The unit's work list is list[lb, lb + n) either way.
template <int ARITH, bool PF>
__device__ __forceinline__ void light_phase(const SketchArgs& a, int64_t lo, int64_t lb, int n, uint64_t Tbits,
                                            float Tf, Reg* regs, uint32_t* map, unsigned char* wbuf, SmemScalars& sh,
                                            Counters& cnt, bool& gave_up, bool ind = false) {
  const bool IND = PF && ind;
  const int tid = threadIdx.x, lane = tid & 31;
  double* wb_r = reinterpret_cast<double*>(wbuf);                 // 1/v of each survivor
  uint32_t* wb_slot = reinterpret_cast<uint32_t*>(wbuf + WB_N * 8);  // its slot in the unit
  int32_t* wb_id = reinterpret_cast<int32_t*>(wbuf + WB_N * 12);     // its id
  const int k = a.k;
  const float kf = (float)k;
  int e = -1, z = 0, msize = 0;
  int32_t id = 0;
  double R = 0.0;
  Fix acc = fix_zero();
  int wcount = 0;
  bool pool_done = false;
  // the warp's next screening batch (PB elements, two per lane when GM_SCREEN_PAIR
  // is 2: independent Philox chains), claimed and loaded one batch ahead so that its
  // weight and id loads are in flight while the current batch is screened
  constexpr int PB = PF ? 32 * GM_SCREEN_PAIR : 32;  // compacted units: GM_SCREEN_PAIR is 1
  int nbase = 0;
  double nv = 0.0, nv2 = 0.0;
  int32_t nid = 0, nid2 = 0;
  int nslot = 0;  // IND: the next batch's element offsets
  if (PF) {
    if (lane == 0) nbase = atomicAdd(&sh.pool, PB);
    nbase = __shfl_sync(FULL, nbase, 0);
    if (nbase + lane < n) {
      if (IND) {
        nslot = (int)__ldcs(a.plist + lb + nbase + lane);
        nv = __ldcs(a.w + lo + nslot);
        nid = __ldcs(a.ids + lo + nslot);
      } else {
        nv = __ldcs(a.w + lo + nbase + lane);
        nid = __ldcs(a.ids + lo + nbase + lane);
      }
    }
    if (PB == 64 && nbase + 32 + lane < n) {
      nv2 = __ldcs(a.w + lo + nbase + 32 + lane);
      nid2 = __ldcs(a.ids + lo + nbase + 32 + lane);
    }
  }
  while (true) {
    // hand survivors to idle lanes, screening new elements while some are idle
    uint32_t nmask = __ballot_sync(FULL, e < 0);
    while (nmask && !(pool_done && wcount == 0)) {
      if (wcount == 0) {
        int base = 0;
        double v = 0.0, v2 = 0.0;
        int32_t idv = 0, idv2 = 0;
        int es = 0;  // IND: the element's offset from lo
        if (PF) {
          base = nbase;
          v = nv;
          idv = nid;
          v2 = nv2;
          idv2 = nid2;
          es = nslot;
        } else {
          if (lane == 0) base = atomicAdd(&sh.pool, 32);
          base = __shfl_sync(FULL, base, 0);
        }
        if (base >= n) {
          pool_done = true;
          break;
        }
        const int slot = IND ? es : base + lane, slot2 = base + 32 + lane;
        const bool in = base + lane < n;
        bool surv = false, surv2 = false;
        if (PF) {
          if (lane == 0) nbase = atomicAdd(&sh.pool, PB);
          nbase = __shfl_sync(FULL, nbase, 0);
          if (nbase + lane < n) {
            if (IND) {
              nslot = (int)__ldcs(a.plist + lb + nbase + lane);
              nv = __ldcs(a.w + lo + nslot);
              nid = __ldcs(a.ids + lo + nslot);
            } else {
              nv = __ldcs(a.w + lo + nbase + lane);
              nid = __ldcs(a.ids + lo + nbase + lane);
            }
          }
          if (PB == 64 && nbase + 32 + lane < n) {
            nv2 = __ldcs(a.w + lo + nbase + 32 + lane);
            nid2 = __ldcs(a.ids + lo + nbase + 32 + lane);
          }
        }
        if (in) {
          if (!PF) v = a.w[lo + slot];
          screen_elem(a, lo, lb, n, slot, v, idv, !PF, Tf, kf, sh, cnt, surv, IND);
        }
        if (PB == 64 && slot2 < n) screen_elem(a, lo, lb, n, slot2, v2, idv2, false, Tf, kf, sh, cnt, surv2);
        const uint32_t sm = __ballot_sync(FULL, surv);
        if (surv) {  // one reciprocal per screening batch, not one per lane refill
          const int p = __popc(sm & lanemask_lt());
          wb_r[p] = arr_rcp<ARITH>(v);
          wb_slot[p] = (uint32_t)slot;
          wb_id[p] = idv;
        }
        wcount = __popc(sm);
        if (PB == 64) {
          const uint32_t sm2 = __ballot_sync(FULL, surv2);
          if (surv2) {
            const int p = wcount + __popc(sm2 & lanemask_lt());
            wb_r[p] = arr_rcp<ARITH>(v2);
            wb_slot[p] = (uint32_t)slot2;
            wb_id[p] = idv2;
          }
          wcount += __popc(sm2);
        }
        __syncwarp();
        continue;
      }
      const int take = min(__popc(nmask), wcount);
      const int rank = __popc(nmask & lanemask_lt());
      if (e < 0 && rank < take) {
        const int q = wcount - 1 - rank;
        e = (int)wb_slot[q];
        id = wb_id[q];
        R = wb_r[q];
        z = 0;
        acc = fix_zero();
        msize = 0;
      }
      wcount -= take;
      __syncwarp();
      nmask = __ballot_sync(FULL, e < 0);
    }
    if (!__any_sync(FULL, e >= 0)) break;  // nothing left to stream
    if (e < 0) continue;
    int J;
    fix_add(acc, arrival_term<ARITH>(id, z, k, a.key0, a.key1, a.ctab, J));
    const uint64_t bb = (uint64_t)__double_as_longlong(arr_mul<ARITH>(fix_round(acc), R));
    ++cnt.arrivals;
    if (bb > Tbits) {  // FastPrune: the rest of this stream is above the bound
      e = -1;
      continue;
    }
    // Fisher-Yates step z on the sparse map (positions < z are final and dropped)
    int iz = -1;
    for (int i = 0; i < msize; ++i)
      if ((map[i * BLOCK + tid] >> 16) == (uint32_t)z) {
        iz = i;
        break;
      }
    uint32_t vz = (uint32_t)z;
    if (iz >= 0) {
      vz = map[iz * BLOCK + tid] & 0xFFFFu;
      --msize;
      map[iz * BLOCK + tid] = map[msize * BLOCK + tid];
    }
    uint32_t c = vz;
    bool overflow = false;
    if (J != z) {
      int ij = -1;
      for (int i = 0; i < msize; ++i)
        if ((map[i * BLOCK + tid] >> 16) == (uint32_t)J) {
          ij = i;
          break;
        }
      if (ij >= 0) {
        c = map[ij * BLOCK + tid] & 0xFFFFu;
        map[ij * BLOCK + tid] = ((uint32_t)J << 16) | vz;
      } else {
        c = (uint32_t)J;
        if (msize >= MAPCAP) {
          overflow = true;
        } else {
          map[msize * BLOCK + tid] = ((uint32_t)J << 16) | vz;
          ++msize;
        }
      }
    }
    if (overflow) {  // restart this element on an 8-lane segment (updates are idempotent)
      a.list[lb + atomicAdd(&sh.hcount, 1)] = (uint32_t)e | TAG_MEDIUM;
      e = -1;
      continue;
    }
    cnt.cas += reg_lower(smem_addr(&regs[c]), bb, (uint64_t)(uint32_t)id, gave_up);
    ++cnt.kept;
    if (++z >= k) e = -1;
  }
}

// FastSearch's release step (Algorithm 1) on the light path: every positive
// element of [lo, lo+n) whose budget grew from bRprev to bR releases the first
// fs_budget(bR) arrivals of its stream (one lane each, from its first arrival:
// register updates are idempotent minima, so re-releasing the earlier ones
// changes nothing); larger budgets go to the work list for the segment phases.
// Elements whose budget did not grow have nothing new to release.
template <int ARITH>
__device__ __forceinline__ void budget_light_phase(const SketchArgs& a, int64_t lo, int n, double bR, double bRprev,
                                                   double bsum, Reg* regs, uint32_t* map, unsigned char* wbuf,
                                                   SmemScalars& sh, Counters& cnt, bool& gave_up) {
  const int tid = threadIdx.x, lane = tid & 31;
  double* wb_r = reinterpret_cast<double*>(wbuf);
  uint32_t* wb_slot = reinterpret_cast<uint32_t*>(wbuf + WB_N * 8);
  int32_t* wb_id = reinterpret_cast<int32_t*>(wbuf + WB_N * 12);
  const int k = a.k;
  int e = -1, z = 0, msize = 0, lim = 0;
  int32_t id = 0;
  double R = 0.0;
  Fix acc = fix_zero();
  int wcount = 0;
  bool pool_done = false;
  while (true) {
    uint32_t nmask = __ballot_sync(FULL, e < 0);
    while (nmask && !(pool_done && wcount == 0)) {
      if (wcount == 0) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&sh.pool, 32);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n) {
          pool_done = true;
          break;
        }
        const int slot = base + lane;
        bool surv = false;
        double v = 0.0;
        int32_t idv = 0;
        if (slot < n) {
          v = a.w[lo + slot];
          if (positive_finite(v)) {
            ++cnt.elements;
            const int b = fs_budget(bR, v, bsum, k), bp = fs_budget(bRprev, v, bsum, k);
            if (b == bp) {
              ++cnt.screened;  // nothing new: its released arrivals are in the registers
            } else if ((float)b > a.light_max) {
              if ((float)b > a.medium_max)
                a.list[lo + n - 1 - atomicAdd(&sh.bcount, 1)] =
                    (uint32_t)slot | ((float)b > a.heavy_max ? TAG_SUPER : TAG_HEAVY);
              else
                a.list[lo + atomicAdd(&sh.hcount, 1)] = (uint32_t)slot | TAG_MEDIUM;
            } else {
              idv = a.ids[lo + slot];
              surv = true;
            }
          }
        }
        const uint32_t sm = __ballot_sync(FULL, surv);
        if (surv) {
          const int p = __popc(sm & lanemask_lt());
          wb_r[p] = arr_rcp<ARITH>(v);
          wb_slot[p] = (uint32_t)slot;
          wb_id[p] = idv;
        }
        wcount = __popc(sm);
        __syncwarp();
        continue;
      }
      const int take = min(__popc(nmask), wcount);
      const int rank = __popc(nmask & lanemask_lt());
      if (e < 0 && rank < take) {
        const int q = wcount - 1 - rank;
        e = (int)wb_slot[q];
        id = wb_id[q];
        R = wb_r[q];
        z = 0;
        acc = fix_zero();
        msize = 0;
        lim = fs_budget(bR, a.w[lo + e], bsum, k);
      }
      wcount -= take;
      __syncwarp();
      nmask = __ballot_sync(FULL, e < 0);
    }
    if (!__any_sync(FULL, e >= 0)) break;
    if (e < 0) continue;
    if (z >= lim) {  // its release is spent
      e = -1;
      continue;
    }
    int J;
    fix_add(acc, arrival_term<ARITH>(id, z, k, a.key0, a.key1, a.ctab, J));
    const uint64_t bb = (uint64_t)__double_as_longlong(arr_mul<ARITH>(fix_round(acc), R));
    ++cnt.arrivals;
    int iz = -1;
    for (int i = 0; i < msize; ++i)
      if ((map[i * BLOCK + tid] >> 16) == (uint32_t)z) {
        iz = i;
        break;
      }
    uint32_t vz = (uint32_t)z;
    if (iz >= 0) {
      vz = map[iz * BLOCK + tid] & 0xFFFFu;
      --msize;
      map[iz * BLOCK + tid] = map[msize * BLOCK + tid];
    }
    uint32_t c = vz;
    bool overflow = false;
    if (J != z) {
      int ij = -1;
      for (int i = 0; i < msize; ++i)
        if ((map[i * BLOCK + tid] >> 16) == (uint32_t)J) {
          ij = i;
          break;
        }
      if (ij >= 0) {
        c = map[ij * BLOCK + tid] & 0xFFFFu;
        map[ij * BLOCK + tid] = ((uint32_t)J << 16) | vz;
      } else {
        c = (uint32_t)J;
        if (msize >= MAPCAP) {
          overflow = true;
        } else {
          map[msize * BLOCK + tid] = ((uint32_t)J << 16) | vz;
          ++msize;
        }
      }
    }
    if (overflow) {  // restart this element on an 8-lane segment
      a.list[lo + atomicAdd(&sh.hcount, 1)] = (uint32_t)e | TAG_MEDIUM;
      e = -1;
      continue;
    }
    if (bb <= DBL_MAX_BITS) {  // an arrival that is not finite takes no register
      cnt.cas += reg_lower(smem_addr(&regs[c]), bb, (uint64_t)(uint32_t)id, gave_up);
      ++cnt.kept;
    }
    if (++z >= k) e = -1;
  }
}

__device__ __forceinline__ void clk_add(Counters&, int which, long long& t) {
  const long long now = read_clock();
  if ((threadIdx.x & 31) == 0) sh_scalars.clk[threadIdx.x >> 5][which] += (unsigned long long)(now - t);
  t = now;
}

// All warp-path classes of one pass: 8-lane segments, then without a barrier
// the 32-lane warps' share of the work list (a warp's hash region is the same
// in both), then the elements promoted out of 8-lane segments, then dense
// permutations (warps < ndense).  (Lowering T to the running y* at the barriers
// saved 2 % of the arrivals and cost more in barriers: measured and dropped.)
// BUDGET: FastSearch's release of budget bR (row sum bsum) instead of the bound.
template <int ARITH, bool BUDGET = false>
// Elements are offsets from lo; the unit's work list and promotions are at lb.
// promote: 8-lane elements that outgrow their table move to the promotion list
// at plist + lb; otherwise they are retagged for the dense path in place (a
// compacted row's warp-path unit, whose plist range holds other entries).
__device__ __forceinline__ void warp_phases(const SketchArgs& a, int64_t lo, int64_t lb, int n, uint64_t Tbits,
                                            Reg* regs, uint32_t* area, uint16_t* dense, SmemScalars& sh,
                                            Counters& cnt, bool& gave_up, long long& t, double bR = 0.0,
                                            double bsum = 0.0, bool promote = true) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nh = sh.hcount, nb = sh.bcount;
  uint32_t* back = a.list + lb + n - nb;  // the 32-lane and dense entries
  {
    const int seg = lane / MED_SW;
    const HashPiN<MED_SLOTS> hp{area + (warp * (32 / MED_SW) + seg) * MED_SLOTS};
    seg_phase<ARITH, MED_SW, HashPiN<MED_SLOTS>, BUDGET>(a, lo, Tbits, regs, a.list + lb, nh, &sh.c_med, TAG_MEDIUM, hp, MED_MAX_FILL,
                             promote ? a.plist + lb : nullptr, &sh.pcount, cnt, gave_up, bR, bsum);
  }
  clk_add(cnt, CLK_MEDIUM, t);
  // a warp's hash region is the same in both phases: the heavy list needs no barrier
  {
    const HashPi hp{area + warp * HASH_SLOTS};
    seg_phase<ARITH, 32, HashPi, BUDGET>(a, lo, Tbits, regs, back, nb, &sh.c_heavy, TAG_HEAVY, hp, HASH_MAX_FILL, nullptr, nullptr,
                         cnt, gave_up, bR, bsum);
  }
  clk_add(cnt, CLK_HEAVY, t);
  __syncthreads();  // every promotion is listed
  clk_add(cnt, CLK_WAIT, t);
  {
    const HashPi hp{area + warp * HASH_SLOTS};
    seg_phase<ARITH, 32, HashPi, BUDGET>(a, lo, Tbits, regs, a.plist + lb, sh.pcount, &sh.c_pheavy, TAG_HEAVY, hp, HASH_MAX_FILL,
                         nullptr, nullptr, cnt, gave_up, bR, bsum);
  }
  clk_add(cnt, CLK_HEAVY, t);
  __syncthreads();
  clk_add(cnt, CLK_WAIT, t);
  // dense permutations: the CTA's own, then as many as fit in the (now idle) hash area
  const int ndense = min(WARPS, a.ndense + (int)(fast_area_bytes() / (pi_stride(a.k) * 2)));
  if (warp < ndense) {
    uint16_t* mine = warp < a.ndense ? dense + (size_t)warp * pi_stride(a.k)
                                     : reinterpret_cast<uint16_t*>(area) + (size_t)(warp - a.ndense) * pi_stride(a.k);
    const DensePi dp{mine};
    seg_phase<ARITH, 32, DensePi, BUDGET>(a, lo, Tbits, regs, back, nb, &sh.c_super, TAG_SUPER, dp, 1 << 30, nullptr, nullptr, cnt,
                         gave_up, bR, bsum);
    seg_phase<ARITH, 32, DensePi, BUDGET>(a, lo, Tbits, regs, a.plist + lb, sh.pcount, &sh.c_psuper, TAG_SUPER, dp, 1 << 30,
                         nullptr, nullptr, cnt, gave_up, bR, bsum);
  }
  clk_add(cnt, CLK_SUPER, t);
  __syncthreads();
  clk_add(cnt, CLK_WAIT, t);
}

__device__ __forceinline__ void reset_lists(SmemScalars& sh) {
  if (threadIdx.x == 0) {
    sh.pool = 0;
    sh.hcount = 0;
    sh.bcount = 0;
    sh.pcount = 0;
    sh.c_med = sh.c_heavy = sh.c_pheavy = sh.c_super = sh.c_psuper = 0;
  }
}

__device__ __forceinline__ void init_regs(const SketchArgs& a, Reg* regs, int k) {
  for (int j = threadIdx.x; j < k; j += BLOCK) {
    if (a.init_y) {  // a running sketch: (+inf, -1) is an unfilled register
      regs[j].y = (uint64_t)__double_as_longlong(a.init_y[j]);
      regs[j].id = a.init_s[j] < 0 ? UNFILLED_ID : (uint64_t)(uint32_t)a.init_s[j];
    } else {
      regs[j].y = INF_BITS;
      regs[j].id = UNFILLED_ID;
    }
  }
}

__device__ __forceinline__ void write_out(const SketchArgs& a, int row, const Reg* regs) {
  const int k = a.k;
  int32_t* s = a.s_out + (int64_t)row * k;
  double* y = a.y_out + (int64_t)row * k;
  for (int j = threadIdx.x; j < k; j += BLOCK) {
    const Reg r = regs[j];
    s[j] = (r.id == UNFILLED_ID) ? -1 : (int32_t)r.id;
    y[j] = __longlong_as_double((long long)r.y);
  }
}

__device__ __forceinline__ void flush_counters(const SketchArgs& a, Counters& cnt, bool gave_up) {
  const int lane = threadIdx.x & 31;
  const uint32_t v32[8] = {cnt.arrivals, cnt.elements, cnt.screened, cnt.heavy,
                           cnt.escalated, cnt.cas, cnt.kept, cnt.fallback};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    unsigned long long v = v32[q];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    if (lane == 0 && v) atomicAdd(&a.hdr->counters[q < 6 ? q : 6 + NCLK + (q - 6)], v);
  }
  if (lane == 0)
    for (int q = 0; q < NCLK; ++q)
      if (sh_scalars.clk[threadIdx.x >> 5][q]) atomicAdd(&a.hdr->counters[6 + q], sh_scalars.clk[threadIdx.x >> 5][q]);
  if (gave_up) atomicOr(&a.hdr->status, WS_ETIMEOUT);
}

// One row (short, or a long row being redone) by one CTA: passes with a growing
// bound from `first_pass` on, until every register is filled.
template <int ARITH>
__device__ __forceinline__ void fastgm_row(const SketchArgs& a, int row, int64_t lo, int n, int first_pass, Reg* regs,
                                           uint32_t* area, uint16_t* dense, unsigned char* wbuf, SmemScalars& sh,
                                           Counters& cnt, bool& gave_up) {
  const int tid = threadIdx.x;
  float sumv;
  int npos;
  long long t = read_clock();
  block_sum<BLOCK>(a, lo, n, sh.red_f, sh.red_i, sumv, npos);
  clk_add(cnt, CLK_SETUP, t);
  for (int pass = first_pass; npos > 0; ++pass) {
    float Tf = a.q2 / sumv;
    if (pass == 0 && !row_bound(a, row, Tf)) Tf = a.q1 / sumv;
    double Td = 0.0;
    bool last = !(Tf < 3.0e38f) || pass >= 12;
    if (!last) {
      Td = f64_from_f32(Tf);
      for (int p = 1; p < pass; ++p) {  // passes >= 2 widen the bound by a.grow each
        Td *= (double)a.grow;
        Tf *= a.grow;  // exact (a power of two): the screen needs Tf = Td as reals, so no clamp below Td
      }
      if (!(Td < 1.0e300) || !(Tf < 3.0e38f)) last = true;
    }
    const uint64_t Tbits = last ? DBL_MAX_BITS : (uint64_t)__double_as_longlong(Td);
    if (last) Tf = __int_as_float(0x7F800000);  // +inf: no screening, everything streams
    reset_lists(sh);
    __syncthreads();
    clk_add(cnt, CLK_SETUP, t);
    light_phase<ARITH, false>(a, lo, lo, n, Tbits, Tf, regs, area, wbuf + (tid >> 5) * WBUF_BYTES, sh, cnt,
                              gave_up);
    clk_add(cnt, CLK_LIGHT, t);
    __syncthreads();
    clk_add(cnt, CLK_WAIT, t);
    warp_phases<ARITH>(a, lo, lo, n, Tbits, regs, area, dense, sh, cnt, gave_up, t);
    // a register above T may still be lowered by an arrival above T: redo wider.
    // (Without a starting sketch that is exactly an unfilled register.)
    int empty = 0;
    for (int j = tid; j < a.k; j += BLOCK) empty |= (regs[j].y > Tbits);
    const bool again = __syncthreads_or(empty) && !last;
    clk_add(cnt, CLK_FINISH, t);
    if (!again) break;
    if (tid == 0) {
      ++cnt.escalated;
      if (pass == 0) ++cnt.fallback;
    }
  }
  write_out(a, row, regs);
  clk_add(cnt, CLK_FINISH, t);
}

// A long row's last finished chunk: read the merged registers; write the row,
// or queue it for a single-CTA redo with a larger bound.
__device__ __forceinline__ void finish_long(const SketchArgs& a, int row, int longi, SmemScalars& sh) {
  const int k = a.k;
  const Reg* g = a.long_regs + (int64_t)longi * k;
  uint64_t Tbits;
  float Tf;
  chunk_bound(a, row, a.longs[longi].sum, Tbits, Tf);
  int empty = 0;
  for (int j = threadIdx.x; j < k; j += BLOCK) empty |= (__ldcg(&g[j].y) > Tbits);
  const bool any_empty = __syncthreads_or(empty) != 0;
  const bool has_pos = a.longs[longi].npos > 0;
  if (any_empty && has_pos && isfinite(a.q_split)) {
    if (threadIdx.x == 0) a.esc[atomicAdd(&a.hdr->esc_count, 1u)] = (uint32_t)row;
    return;
  }
  int32_t* s = a.s_out + (int64_t)row * k;
  double* y = a.y_out + (int64_t)row * k;
  for (int j = threadIdx.x; j < k; j += BLOCK) {
    const uint64_t yb = __ldcg(&g[j].y), id = __ldcg(&g[j].id);
    s[j] = (id == UNFILLED_ID) ? -1 : (int32_t)id;
    y[j] = __longlong_as_double((long long)yb);
  }
}

// Bound of pass `pass` of a bound-free long-row chunk: FastSearch's doubling
// horizon 2^pass / (the chunk's sum), unless the row's merged registers g are all
// filled, when their largest value y* (rounded up to FP32) is used instead if
// smaller: every final register of the row is at most y*, so no arrival above it
// can matter (FastPrune), and that pass is the chunk's last (returns true).
// Block-wide (barriers); every thread gets the same result.
__device__ __forceinline__ bool ladder_bound(const Reg* g, int k, float sumc, int pass, SmemScalars& sh,
                                             uint64_t& Tbits, float& Tf) {
  unsigned long long m = 0ull;
  for (int j = threadIdx.x; j < k; j += BLOCK) {
    const unsigned long long y = __ldcg(&g[j].y);
    m = y > m ? y : m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(FULL, m, d);
    m = o > m ? o : m;
  }
  unsigned long long* red = reinterpret_cast<unsigned long long*>(sh.red_d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0ull;
  for (int q = 0; q < WARPS; ++q) m = red[q] > m ? red[q] : m;
  __syncthreads();
  float T = __int_as_float(0x7F800000);
  if (pass < 40) T = ldexpf(1.0f, pass) / sumc;  // beyond: no bound at all
  bool final = !(T < 3.0e38f);
  if (m < INF_BITS) {  // every register of the row is filled: FastPrune by its y*
    const float ty = fmaxf(__double2float_ru(__longlong_as_double((long long)m)), 1.17549435e-38f);
    if (ty <= T) {
      T = ty;
      final = true;
    }
  }
  const bool none = !(T < 3.0e38f);
  Tbits = none ? DBL_MAX_BITS : (uint64_t)__double_as_longlong(f64_from_f32(T));
  Tf = none ? __int_as_float(0x7F800000) : T;
  return final;
}

// One row by one CTA under the paper's FastSearch schedule (Algorithm 1): rounds
// R = Delta, 2 Delta, ... release each element's first ceil(R v / sum v) arrivals
// (sum v in FP64, a fixed order) until every register holds an arrival; then
// FastPrune: every element streams up to the row's y* = max_j y_j (arrivals equal
// to y* still take part in the tie rule).  After FS_MAX_ROUNDS rounds a last one
// releases every arrival.  Writes the row and the number of rounds it took.
template <int ARITH>
__device__ __forceinline__ void fastsearch_row(const SketchArgs& a, int row, int64_t lo, int n, Reg* regs,
                                               uint32_t* area, uint16_t* dense, unsigned char* wbuf,
                                               SmemScalars& sh, Counters& cnt, bool& gave_up) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float sumv;
  int npos;
  long long t = read_clock();
  block_sum<BLOCK>(a, lo, n, sh.red_f, sh.red_i, sumv, npos);
  const double dsum = block_dsum<BLOCK>(a.w, lo, n, sh.red_d);
  int rounds = 0;
  if (npos > 0) {
    for (int r = 1;; ++r) {
      const bool all = r > FS_MAX_ROUNDS;
      const double bR = all ? __longlong_as_double((long long)INF_BITS) : (double)r * (double)a.fs_delta;
      const double bRprev = (double)(r - 1) * (double)a.fs_delta;
      reset_lists(sh);
      __syncthreads();
      budget_light_phase<ARITH>(a, lo, n, bR, bRprev, dsum, regs, area, wbuf + (tid >> 5) * WBUF_BYTES, sh, cnt,
                                gave_up);
      __syncthreads();
      warp_phases<ARITH, true>(a, lo, lo, n, DBL_MAX_BITS, regs, area, dense, sh, cnt, gave_up, t, bR, dsum);
      rounds = r;
      int empty = 0;
      for (int j = tid; j < a.k; j += BLOCK) empty |= (regs[j].y == INF_BITS);
      if (!__syncthreads_or(empty) || all) break;
    }
    // FastPrune by the row's y*
    unsigned long long m = 0ull;
    for (int j = tid; j < a.k; j += BLOCK) m = regs[j].y > m ? regs[j].y : m;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const unsigned long long o = __shfl_xor_sync(FULL, m, d);
      m = o > m ? o : m;
    }
    unsigned long long* red = reinterpret_cast<unsigned long long*>(sh.red_d);
    if (lane == 0) red[warp] = m;
    __syncthreads();
    m = 0ull;
    for (int q = 0; q < WARPS; ++q) m = red[q] > m ? red[q] : m;
    __syncthreads();
    if (m < INF_BITS) {
      const float Tf = fmaxf(__double2float_ru(__longlong_as_double((long long)m)), 1.17549435e-38f);
      reset_lists(sh);
      __syncthreads();
      light_phase<ARITH, false>(a, lo, lo, n, m, Tf, regs, area, wbuf + (tid >> 5) * WBUF_BYTES, sh, cnt, gave_up);
      __syncthreads();
      warp_phases<ARITH>(a, lo, lo, n, m, regs, area, dense, sh, cnt, gave_up, t);
    }
  }
  write_out(a, row, regs);
  if (tid == 0) {
    if (a.fs_rounds) a.fs_rounds[row] = rounds;
    if (rounds > 1) cnt.escalated += (uint32_t)(rounds - 1);
  }
}

// One chunk of a long row: its elements with the bound from the row's sum (or,
// in the bound-free mode, a ladder of passes on the chunk's own registers), then
// its registers merged into the row's global ones.
// One element's arrival stream by the whole CTA (Sec. 2.2; a super-heavy element
// of a compacted long row, whose stream would otherwise be one warp's long serial
// chain): rounds of BLOCK consecutive arrivals, each thread one arrival's term and
// RandInt target in parallel; the exact prefix sums by warp scans and a scan of
// the warps' totals (carried across rounds); the arrivals up to the first above T
// kept (times ascend, so they are a prefix); their Fisher-Yates steps on a dense
// permutation by warp 0, 32 steps at a time in order; then each thread lowers its
// arrival's register.  Block-wide.  Scratch: area (targets, servers, warp
// totals), pi (k entries).
template <int ARITH>
__device__ __forceinline__ void coop_stream(const SketchArgs& a, int64_t lo, uint32_t slot, uint64_t Tbits, Reg* regs,
                                         uint32_t* area, uint16_t* pi, Counters& cnt, bool& gave_up) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k;
  uint16_t* Jb = reinterpret_cast<uint16_t*>(area);             // BLOCK targets
  uint16_t* cb = Jb + BLOCK;                                      // BLOCK servers
  Fix* tot = reinterpret_cast<Fix*>(area + BLOCK);                // WARPS totals, then offsets; [WARPS]: carry
  const int32_t id = a.ids[lo + slot];
  const double R = arr_rcp<ARITH>(a.w[lo + slot]);
  const DensePi dp{pi};
  dp.reset_seg(k, tid, BLOCK);
  if (tid == 0) tot[WARPS] = fix_zero();
  __syncthreads();
  for (int z0 = 0; z0 < k; z0 += BLOCK) {
    const int z = z0 + tid;
    Fix f = fix_zero();
    int J = z;
    if (z < k) f = arrival_term<ARITH>(id, z, k, a.key0, a.key1, a.ctab, J);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Fix g;
      g.w0 = __shfl_up_sync(FULL, f.w0, d);
      g.w1 = __shfl_up_sync(FULL, f.w1, d);
      if (lane >= d) fix_add(f, g);
    }
    if (lane == 31) tot[warp] = f;
    Jb[tid] = (uint16_t)(z < k ? J : 0);
    __syncthreads();
    if (warp == 0) {  // offsets of the warps: the carry plus the exclusive scan of their totals
      Fix x = lane < WARPS ? tot[lane] : fix_zero();
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        Fix g;
        g.w0 = __shfl_up_sync(FULL, x.w0, d);
        g.w1 = __shfl_up_sync(FULL, x.w1, d);
        if (lane >= d) fix_add(x, g);
      }
      Fix e;  // exclusive: the lane below's inclusive sum
      e.w0 = __shfl_up_sync(FULL, x.w0, 1);
      e.w1 = __shfl_up_sync(FULL, x.w1, 1);
      if (lane == 0) e = fix_zero();
      const Fix c = tot[WARPS];
      fix_add(e, c);
      __syncwarp();
      if (lane < WARPS) tot[lane] = e;
    }
    __syncthreads();
    fix_add(f, tot[warp]);  // the exact prefix sum through arrival z
    const uint64_t bb = z < k ? (uint64_t)__double_as_longlong(arr_mul<ARITH>(fix_round(f), R)) : ~0ull;
    const bool keep = bb <= Tbits;
    const int nk = __syncthreads_count(keep);
    if (tid == BLOCK - 1) tot[WARPS] = f;  // the next round's carry (read after the barriers below)
    if (warp == 0) {  // Fisher-Yates steps z0 .. z0 + nk - 1, in order
      for (int s0 = 0; s0 < nk; s0 += 32) {
        const int n = min(32, nk - s0);
        const int Jl = lane < n ? (int)Jb[s0 + lane] : z0 + s0 + lane;
        int c;
        seg_fy_steps<32>(dp, z0 + s0, Jl, n, lane, c);
        if (lane < n) cb[s0 + lane] = (uint16_t)c;
      }
    }
    __syncthreads();
    if (keep) {
      cnt.cas += reg_lower(smem_addr(&regs[cb[tid]]), bb, (uint64_t)(uint32_t)id, gave_up);
      ++cnt.kept;
    }
    if (tid == 0) cnt.arrivals += (uint32_t)min(BLOCK, k - z0);
    __syncthreads();  // Jb, cb and the totals are reused
    if (nk < BLOCK) break;
  }
  if (tid == 0) ++cnt.heavy;
}

// CMP: compiled with the compacted units (taken when the launch compacted its
// long rows, a.compact).
template <int ARITH, bool CMP>
__device__ __forceinline__
void chunk_unit(const SketchArgs& a, int row, int chunk, int longi, int64_t lo, int64_t hi, Reg* regs,
                uint32_t* area, uint16_t* dense, unsigned char* wbuf, SmemScalars& sh, Counters& cnt,
                bool& gave_up) {
  const int k = a.k, tid = threadIdx.x;
  Reg* g = a.long_regs + (int64_t)longi * k;
  const int nsuper = CMP && chunk < 0 ? (int)a.longs[longi].nsuper : 0;  // chunk < 0: compacted units only
  if (CMP && chunk < 0 && -1 - chunk < nsuper) {  // a super-heavy element of a compacted row: the whole CTA
    long long t = read_clock();
    uint64_t Tbits;
    float Tf;
    chunk_bound(a, row, a.longs[longi].sum, Tbits, Tf);
    coop_stream<ARITH>(a, lo, a.plist[hi - 1 - (-1 - chunk)], Tbits, regs, area, dense, cnt, gave_up);
    clk_add(cnt, CLK_SUPER, t);
    merge_to_global<BLOCK>(regs, g, k, gave_up);
    return;
  }
  // A unit of heavy elements of a compacted row: entries list[hi - j1, hi - j0)
  // on the warp paths only.  A unit of a compacted row's compact list: entries
  // [c0, c1), offsets from lo, one pass at the row's bound.  Otherwise elements
  // [clo, chi) of the row.
  const bool heavy = CMP && chunk < 0, cmp = CMP && a.compact != 0;
  int64_t clo, lb, chi;
  if (heavy) {
    const int64_t j0 = (int64_t)(-1 - chunk - nsuper) * HEAVY_UNIT;
    const int64_t j1 = min((int64_t)a.longs[longi].nheavy, j0 + HEAVY_UNIT);
    clo = lo;
    lb = hi - j1;
    chi = lo + j1 - j0;
  } else if (cmp) {
    const int64_t cu = a.hdr->cunit;
    const int64_t c0 = (int64_t)chunk * cu;
    clo = lo;
    lb = lo + c0;
    chi = lo + min((int64_t)a.longs[longi].ncomp, c0 + cu) - c0;
  } else {
    clo = lo + (int64_t)chunk * a.chunk_len;
    lb = clo;
    chi = min(hi, clo + a.chunk_len);
  }
  if (chi > clo) {
    float tdummy;
    const bool ladder = !cmp && a.chunk_ladder && !row_bound(a, row, tdummy);
    float sumc = 0.0f;
    int nposc = 1;
    long long t = read_clock();
    if (ladder) block_sum<BLOCK>(a, clo, (int)(chi - clo), sh.red_f, sh.red_i, sumc, nposc);
    for (int pass = 0; nposc > 0; ++pass) {
      uint64_t Tbits;
      float Tf;
      bool final = true;
      if (ladder)
        final = ladder_bound(g, k, sumc, pass, sh, Tbits, Tf);
      else
        chunk_bound(a, row, a.longs[longi].sum, Tbits, Tf);
      reset_lists(sh);
      if (heavy && tid == 0) {  // the whole unit is both its front (8-lane) and back (32-lane) list
        sh.bcount = (int)(chi - clo);
        sh.hcount = GM_SPLIT_MEDIUM ? (int)(chi - clo) : 0;
      }
      __syncthreads();
      clk_add(cnt, CLK_SETUP, t);
      if (!heavy) {
        light_phase<ARITH, true>(a, clo, lb, (int)(chi - clo), Tbits, Tf, regs, area,
                                 wbuf + (tid >> 5) * WBUF_BYTES, sh, cnt, gave_up, cmp);
        clk_add(cnt, CLK_LIGHT, t);
        __syncthreads();
        clk_add(cnt, CLK_WAIT, t);
      }
      warp_phases<ARITH>(a, clo, lb, (int)(chi - clo), Tbits, regs, area, dense, sh, cnt, gave_up, t, 0.0, 0.0,
                         !heavy);
      if (final) break;
      // the chunk's own sketch is exact once its registers are all at or below T
      int empty = 0;
      for (int j = tid; j < k; j += BLOCK) empty |= (regs[j].y > Tbits);
      if (!__syncthreads_or(empty)) break;
      if (tid == 0) ++cnt.escalated;
    }
    merge_to_global<BLOCK>(regs, g, k, gave_up);
  }
}

template <int ARITH, int MODE>
__global__ void __launch_bounds__(BLOCK, CTAS_PER_SM) fastgm_kernel(SketchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemScalars& sh = sh_scalars;
  const int k = a.k;
  Reg* regs = reinterpret_cast<Reg*>(smem);
  uint32_t* area = reinterpret_cast<uint32_t*>(smem + (size_t)k * sizeof(Reg));
  uint16_t* dense = reinterpret_cast<uint16_t*>(smem + (size_t)k * sizeof(Reg) + fast_area_bytes());
  unsigned char* wbuf = smem + (size_t)k * sizeof(Reg) + fast_area_bytes() + (size_t)a.ndense * pi_stride(k) * 2;
  const int tid = threadIdx.x;
  Counters cnt;
  cnt.zero();
  bool gave_up = false;
  const long long t_start = read_clock();
  if ((tid & 31) == 0)
    for (int q = 0; q < NCLK; ++q) sh.clk[tid >> 5][q] = 0ull;
  const uint32_t n_extra = a.hdr->n_extra, n_long = a.hdr->n_long, n_hu = a.hdr->n_hunits;
  const uint32_t n_units = (MODE == MODE_MAIN || MODE == MODE_CMP) ? n_hu + n_extra + (uint32_t)a.n_rows
                           : MODE == MODE_FS ? (uint32_t)a.n_rows
                                             : a.hdr->esc_count;

  while (true) {
    if (tid == 0) sh.unit = (int)atomicAdd(MODE == MODE_ESC ? &a.hdr->esc_counter : &a.hdr->unit_counter, 1u);
    __syncthreads();
    const uint32_t u = (uint32_t)sh.unit;
    if (u >= n_units) break;
    int row, chunk, longi;
    if (MODE == MODE_ESC) {
      row = (int)a.esc[u];
      chunk = 0;
      longi = -1;
    } else if (MODE == MODE_FS) {
      row = (int)u;
      chunk = 0;
      longi = -1;
    } else {
      resolve_unit(a, u, n_hu, n_extra, n_long, row, chunk, longi);
    }
    int64_t lo, hi;
    row_bounds(a, row, lo, hi);
    init_regs(a, regs, k);
    if constexpr (MODE == MODE_FS) {
      fastsearch_row<ARITH>(a, row, lo, (int)(hi - lo), regs, area, dense, wbuf, sh, cnt, gave_up);
      __syncthreads();
      continue;
    }
    if (longi < 0) {  // the whole row in this CTA
      fastgm_row<ARITH>(a, row, lo, (int)(hi - lo), MODE == MODE_ESC ? 1 : 0, regs, area, dense, wbuf, sh, cnt,
                        gave_up);
      __syncthreads();
      continue;
    }
    if (a.longs[longi].npos > 0)
      chunk_unit<ARITH, MODE == MODE_CMP || SHARED_CMP>(a, row, chunk, longi, lo, hi, regs, area, dense, wbuf, sh,
                                                        cnt, gave_up);
    __threadfence();
    __syncthreads();
    if (tid == 0)
      sh.last = (atomicAdd(&a.longs[longi].done, 1u) == a.longs[longi].nchunks + a.longs[longi].nhunits - 1u) ? 1 : 0;
    __syncthreads();
    if (sh.last) {
      __threadfence();
      finish_long(a, row, longi, sh);
    }
    __syncthreads();
  }
  if ((tid & 31) == 0) sh_scalars.clk[tid >> 5][CLK_TOTAL] += (unsigned long long)(read_clock() - t_start);
  __syncwarp();
  flush_counters(a, cnt, gave_up);
}

// The plain sketch: every positive element, all k arrivals, warp path with one
// dense permutation per warp.  Long rows are chunked and merged like FastGM's.
template <int ARITH>
__global__ void __launch_bounds__(BLOCK, 1) plain_kernel(SketchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemScalars& sh = sh_scalars;
  const int k = a.k;
  Reg* regs = reinterpret_cast<Reg*>(smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const DensePi dp{reinterpret_cast<uint16_t*>(smem + (size_t)k * sizeof(Reg)) + (size_t)warp * pi_stride(k)};
  Counters cnt;
  cnt.zero();
  bool gave_up = false;
  const uint32_t n_extra = a.hdr->n_extra, n_long = a.hdr->n_long;
  const uint32_t n_units = n_extra + (uint32_t)a.n_rows;
  while (true) {
    if (tid == 0) sh.unit = (int)atomicAdd(&a.hdr->unit_counter, 1u);
    __syncthreads();
    const uint32_t u = (uint32_t)sh.unit;
    if (u >= n_units) break;
    int row, chunk, longi;
    resolve_unit(a, u, 0u, n_extra, n_long, row, chunk, longi);
    int64_t lo, hi;
    row_bounds(a, row, lo, hi);
    init_regs(a, regs, k);
    const int64_t clo = longi < 0 ? lo : lo + (int64_t)chunk * a.chunk_len;
    const int64_t chi = longi < 0 ? hi : min(hi, clo + a.chunk_len);
    const int n = (int)(chi - clo);
    if (longi < 0) {
      float sumv;
      int npos;
      block_sum<BLOCK>(a, lo, n, sh.red_f, sh.red_i, sumv, npos);  // validation only
    }
    // budget pass (FastSearch, Algorithm 1): element i releases ceil(R v_i / sum v)
    // of its arrivals, the ratio and product in FP64 as the paper's schedule states
    double Rr = 0.0, dsum = 0.0;
    if (a.r_row) {
      Rr = a.r_row[row];
      dsum = longi < 0 ? block_dsum<BLOCK>(a.w, lo, n, sh.red_d) : __ldcg(&a.longs[longi].dsum);
    }
    if (tid == 0) sh.pool = 0;
    __syncthreads();
    while (true) {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(&sh.pool, 1);
      slot = __shfl_sync(FULL, slot, 0);
      if (slot >= n) break;
      const double v = a.w[clo + slot];
      if (!positive_finite(v)) continue;
      if (lane == 0) ++cnt.elements;
      const int32_t id = a.ids[clo + slot];
      const double R = arr_rcp<ARITH>(v);
      int lim = k;
      if (a.r_row) {
        const double b = ceil(__dmul_rn(Rr, __ddiv_rn(v, dsum)));
        lim = b < (double)k ? (int)b : k;
      }
      dp.reset(k, lane);
      Fix carry = fix_zero();
      for (int z0 = 0; z0 < lim; z0 += 32) {  // all k arrivals (or the budget), 32 per step
        int J, c;
        const uint64_t bb = warp_batch<ARITH>(id, R, z0, k, a.key0, a.key1, a.ctab, carry, lane, J);
        const int nz = min(32, lim - z0);
        if (lane == 0) cnt.arrivals += (uint32_t)nz;
        warp_fy_steps(dp, z0, J, nz, lane, c);
        if (lane < nz && bb <= DBL_MAX_BITS) {
          cnt.cas += reg_lower(smem_addr(&regs[c]), bb, (uint64_t)(uint32_t)id, gave_up);
          ++cnt.kept;
        }
      }
    }
    __syncthreads();
    if (longi < 0) {
      write_out(a, row, regs);
      __syncthreads();
      continue;
    }
    merge_to_global<BLOCK>(regs, a.long_regs + (int64_t)longi * k, k, gave_up);
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.last = (atomicAdd(&a.longs[longi].done, 1u) == a.longs[longi].nchunks - 1) ? 1 : 0;
    __syncthreads();
    if (sh.last) {
      __threadfence();
      const Reg* gg = a.long_regs + (int64_t)longi * k;
      for (int j = tid; j < k; j += BLOCK) {
        const uint64_t yb = __ldcg(&gg[j].y), id = __ldcg(&gg[j].id);
        a.s_out[(int64_t)row * k + j] = (id == UNFILLED_ID) ? -1 : (int32_t)id;
        a.y_out[(int64_t)row * k + j] = __longlong_as_double((long long)yb);
      }
    }
    __syncthreads();
  }
  flush_counters(a, cnt, gave_up);
}

// Dense permutations per CTA: as many as fit with CTAS_PER_SM CTAs per SM (at least one).
static int dense_buffers(int k, size_t smem_per_sm) {
  const size_t budget = smem_per_sm / CTAS_PER_SM - 2048;  // each CTA with ~1 KB reserved and static smem
  const size_t base = fast_smem_bytes(k, 0);
  if (budget <= base + pi_stride(k) * 2) return 1;
  const size_t n = (budget - base) / (pi_stride(k) * 2);
  return (int)(n < 1 ? 1 : (n > (size_t)WARPS ? (size_t)WARPS : n));
}

template <class KERNEL>
static int occupancy_grid(KERNEL kern, size_t sm, int nsm, int cap, int& grid) {
  int per_sm = 0;
  if (allow_max_smem((const void*)kern) != GM_OK) return GM_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, sm) != cudaSuccess) return GM_ECUDA;
  if (per_sm < 1) return GM_EINVAL;
  grid = nsm * per_sm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  return GM_OK;
}

// Elements per chunk of a long row for a launch of `grid` persistent CTAs: about
// 1.75 units per CTA if the batch were all long rows, in whole 4,096-element
// steps, between 8,192 and GM_CHUNK_LEN.  A batch of many long rows gets large
// chunks (each unit pays phase barriers, the tails of its heavy elements and a
// merge: 16 x 10^6 Pareto(1.2) at k = 4096, per main-kernel launch: 32K chunks 0.400
// ms, 48K 0.383, 64K 0.373, 112K 0.426); a single long row (a Stream-FastGM chunk
// of 10^6 items) gets small ones, so that its units still fill the grid.
static int chunk_len_for(int64_t nnz, int grid) {
  int64_t c = (int64_t)((double)nnz / (GM_CHUNK_UNITS_PER_CTA * (double)(grid > 0 ? grid : 1)));
  c = (c + 4095) / 4096 * 4096;
  if (c < 8192) c = 8192;
  if (c > GM_CHUNK_LEN) c = GM_CHUNK_LEN;
  return (int)c;
}

template <int ARITH>
static int launch_all(SketchArgs a, bool plain, int nsm, cudaStream_t stream) {
  const size_t sm = plain ? plain_smem_bytes(a.k) : fast_smem_bytes(a.k, a.ndense);
  int grid = 0, rc;
  // The plain sketch keeps SPLIT_LEN-element chunks: every element costs k arrivals
  // there, so a 64K chunk on one CTA would set the launch's tail (0.49 s against
  // 0.41 s at k = 1024 on the lognormal batch).
  if (plain) {
    a.chunk_len = SPLIT_LEN;
  } else {
    int per_sm = 0;
    if (allow_max_smem((const void*)fastgm_kernel<ARITH, MODE_MAIN>) != GM_OK) return GM_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fastgm_kernel<ARITH, MODE_MAIN>, BLOCK, sm) !=
        cudaSuccess)
      return GM_ECUDA;
    a.chunk_len = chunk_len_for(a.nnz, nsm * (per_sm > 0 ? per_sm : 1));
  }
  // Long rows with a fixed bound (closed form, learned or caller-given) are
  // compacted: screened first by the whole grid, then sketched from their lists.
  // The bound-free ladder grows each chunk's bound, so it keeps the element ranges.
  // (Compact entries are offsets within the row, tagged in the work lists' top two
  // bits: rows must stay below 2^30 elements, which nnz < 2^30 ensures.)
  // Only large batches of long rows (an average row of more than SPLIT_LEN
  // elements, more than 2^23 elements in all) are compacted: a few long rows
  // among many short ones overlap their chunk units with the short rows; a batch
  // of one or two long rows has too few compacted units to fill the GPU (a
  // serving batch with a 4.5 x 10^6-element row was slower compacted); and a
  // Stream-FastGM chunk (one row from a running sketch, whose y* screens out most
  // of it) gains less from a second pass over its few survivors than it costs.
  a.compact = (GM_COMPACT_LONG && GM_SCREEN_PAIR == 1 && !plain && a.fs_delta == 0 && !a.chunk_ladder &&
               !a.init_y && a.nnz < ((int64_t)1 << 30) &&
               ((a.flags & GM_FLAG_COMPACT_LONG) ||
                (a.nnz > ((int64_t)1 << 23) && a.nnz > (int64_t)SPLIT_LEN * a.n_rows)))
                  ? 1
                  : 0;
  const int max_units = a.n_rows + (int)((a.nnz + a.chunk_len - 1) / a.chunk_len) + a.max_long +
                        (a.compact ? (int)(a.nnz / 2048) : 0);
  if (a.fs_delta == 0) {  // FastSearch's schedule takes every row whole: no long-row plan
    plan_kernel<<<1, PLAN_THREADS, 0, stream>>>(a);
    longprep_kernel<<<nsm * 8, PREP_THREADS, 0, stream>>>(a);
  }
  if (plain) {
    if constexpr (BLOCK != 512) {
      return GM_EINVAL;  // the plain sketch runs with 512-thread CTAs only
    } else {
      rc = occupancy_grid(plain_kernel<ARITH>, sm, nsm, max_units, grid);
      if (rc != GM_OK) return rc;
      if (g_main_before) cudaEventRecord(g_main_before, stream);
      plain_kernel<ARITH><<<grid, BLOCK, sm, stream>>>(a);
      if (g_main_after) cudaEventRecord(g_main_after, stream);
      return GM_OK;
    }
  }
  if (a.fs_delta > 0) {  // FastSearch's schedule: every row whole, no chunks, no redo kernel
    rc = occupancy_grid(fastgm_kernel<ARITH, MODE_FS>, sm, nsm, a.n_rows, grid);
    if (rc != GM_OK) return rc;
    if (g_main_before) cudaEventRecord(g_main_before, stream);
    fastgm_kernel<ARITH, MODE_FS><<<grid, BLOCK, sm, stream>>>(a);
    if (g_main_after) cudaEventRecord(g_main_after, stream);
    return GM_OK;
  }
  bool launched = false;
  if constexpr (!SHARED_CMP) {
    if (a.compact) {  // the same persistent kernel, compiled with the compacted units
      rc = occupancy_grid(fastgm_kernel<ARITH, MODE_CMP>, sm, nsm, max_units, grid);
      if (rc != GM_OK) return rc;
      screen_kernel<<<nsm * 8, SCREEN_THREADS, 0, stream>>>(a);
      compact_plan_kernel<<<1, PLAN_THREADS, 0, stream>>>(a, grid);
      if (g_main_before) cudaEventRecord(g_main_before, stream);
      fastgm_kernel<ARITH, MODE_CMP><<<grid, BLOCK, sm, stream>>>(a);
      if (g_main_after) cudaEventRecord(g_main_after, stream);
      launched = true;
    }
  }
  if (!launched) {
    rc = occupancy_grid(fastgm_kernel<ARITH, MODE_MAIN>, sm, nsm, max_units, grid);
    if (rc != GM_OK) return rc;
    if (a.compact) {
      screen_kernel<<<nsm * 8, SCREEN_THREADS, 0, stream>>>(a);
      compact_plan_kernel<<<1, PLAN_THREADS, 0, stream>>>(a, grid);
    }
    if (g_main_before) cudaEventRecord(g_main_before, stream);
    fastgm_kernel<ARITH, MODE_MAIN><<<grid, BLOCK, sm, stream>>>(a);
    if (g_main_after) cudaEventRecord(g_main_after, stream);
  }
  // the redo kernel: long rows left unfilled are rare (p = 1e-3 per row), so a
  // small grid; its empty launch then costs little
  int grid_esc = 0;
  rc = occupancy_grid(fastgm_kernel<ARITH, MODE_ESC>, sm, nsm, a.max_long < 16 ? a.max_long : 16, grid_esc);
  if (rc != GM_OK) return rc;
  fastgm_kernel<ARITH, MODE_ESC><<<grid_esc, BLOCK, sm, stream>>>(a);
  return GM_OK;
}

// The whole launch for this shape: dense permutations that fit, then the kernels.
template <int ARITH>
int launch(SketchArgs a, bool plain, int nsm, size_t smem_per_sm, cudaStream_t stream) {
  a.ndense = dense_buffers(a.k, smem_per_sm);
  return launch_all<ARITH>(a, plain, nsm, stream);
}

}  // namespace GM_SHAPE_NS
