// Grid-wide barrier of a cooperative launch, with a wall-clock limit.
//
// Arrival is a release-add on a counter that only grows; a block waits until
// the counter reaches epoch * nblk, polling with acquire loads.  The wait gives up after spin_ns of wall-clock time, or as
// soon as another block has given up (the shared timeout word), and then
// reports failure instead of hanging.
#pragma once

namespace cgp {

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One 128-bit access: a single memory operation (no tearing between the halves).
__device__ __forceinline__ void st_relaxed_b128(void* p, unsigned long long lo, unsigned long long hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tmov.b128 t, {%1, %2};\n\tst.relaxed.gpu.global.b128 [%0], t;\n\t}" ::"l"(p),
               "l"(lo), "l"(hi)
               : "memory");
}

__device__ __forceinline__ ulonglong2 ld_relaxed_b128(const void* p) {
  unsigned long long lo, hi;
  asm volatile("{\n\t.reg .b128 t;\n\tld.relaxed.gpu.global.b128 t, [%2];\n\tmov.b128 {%0, %1}, t;\n\t}"
               : "=l"(lo), "=l"(hi)
               : "l"(p)
               : "memory");
  return make_ulonglong2(lo, hi);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One thread: wait until the word at p (which only grows) reaches target,
// polling with acquire loads (the load that sees it is itself the acquire,
// so no further round trip follows); false when the wait gave up after
// spin_ns of wall-clock time or because another block gave up first.
__device__ __forceinline__ bool wait_at_least(const unsigned* p, unsigned target, int* timeout, long long spin_ns) {
  unsigned long long t0 = 0;
  unsigned spins = 0;
  while (ld_acquire(p) < target) {
    if ((++spins & 127u) == 0) {
      if (*(volatile int*)timeout) return false;
      const unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else if ((long long)(now - t0) > spin_ns) {
        atomicExch(timeout, 1);
        return false;
      }
    }
  }
  return true;
}

// Thread 0 of the block: wait for the `epoch`-th completion of the barrier
// over nblk blocks (after this block's arrival); returns false when the wait
// gave up.
__device__ __forceinline__ bool barrier_wait(unsigned* bar, int* timeout, unsigned nblk, unsigned epoch,
                                             long long spin_ns) {
  return wait_at_least(bar, epoch * nblk, timeout, spin_ns);
}

// Thread 0 of the block: arrive, then wait as above.
__device__ __forceinline__ bool barrier_arrive_wait(unsigned* bar, int* timeout, unsigned nblk, unsigned epoch,
                                                    long long spin_ns) {
  red_release_add(bar, 1u);
  return barrier_wait(bar, timeout, nblk, epoch, spin_ns);
}

}  // namespace cgp
