// Host-only check of the stream-K split used by the pair sweeps: for many shapes,
// walking each block's units the way the kernels do covers every (target tile,
// source unit) exactly once, slots b + t never collide, and the reducer's test of
// "block b ran a unit of tile t" matches the walk.  Prints "OK" or the failure.
#include <stdio.h>
#include <set>
#include <vector>

#include "vpm_common.cuh"

using vpm::StreamK;

static int check(int TT, int np, int ns, int wp, int ws, int B)
{
    StreamK sk;
    sk.TT = TT, sk.np = np, sk.ns = ns, sk.wp = wp, sk.ws = ws;
    sk.C = (long long)np * wp + (long long)ns * ws;
    sk.tot = (long long)TT * sk.C;
    sk.B = B;
    const int nu = np + ns;
    std::vector<int> seen((size_t)TT * nu, 0);
    std::set<long long> slots;
    std::vector<std::set<int>> wrote(TT);
    for (int b = 0; b < B; ++b) {
        const long long lo = sk.lo(b), hi = sk.lo(b + 1);
        int t, k;
        sk.first_at_or_after(lo, t, k);
        if (t >= TT || sk.unit_start(t, k) >= hi) continue;
        for (;;) {
            seen[(size_t)t * nu + k]++;
            if (sk.block_of(sk.unit_start(t, k)) != b) {
                printf("block_of mismatch b=%d t=%d k=%d\n", b, t, k);
                return 1;
            }
            int nt = t, nk = k + 1;
            if (nk == nu) nk = 0, ++nt;
            const bool has_next = nt < TT && sk.unit_start(nt, nk) < hi;
            if (!has_next || nt != t) {
                if (!slots.insert((long long)b + t).second) {
                    printf("slot collision b=%d t=%d\n", b, t);
                    return 1;
                }
                wrote[t].insert(b);
            }
            if (!has_next) break;
            t = nt, k = nk;
        }
    }
    for (size_t i = 0; i < seen.size(); ++i)
        if (seen[i] != 1) {
            printf("unit %zu seen %d times (TT=%d np=%d ns=%d B=%d)\n", i, seen[i], TT, np, ns, B);
            return 1;
        }
    for (int t = 0; t < TT; ++t) {
        const int b0 = sk.block_of(sk.unit_start(t, 0)), b1 = sk.block_of(sk.unit_start(t, nu - 1));
        std::set<int> found;
        for (int b = b0; b <= b1; ++b) {
            const long long lo = sk.lo(b), hi = sk.lo(b + 1);
            const long long c0 = lo > (long long)t * sk.C ? lo : (long long)t * sk.C;
            int tt, kk;
            sk.first_at_or_after(c0, tt, kk);
            if (tt != t || sk.unit_start(tt, kk) >= hi) continue;
            found.insert(b);
        }
        if (found != wrote[t]) {
            printf("reducer set mismatch at t=%d\n", t);
            return 1;
        }
        if (b1 >= B + 0 && b1 != B - 1) {
            printf("block range overflow\n");
            return 1;
        }
        if ((long long)b1 + t >= (long long)TT + B) {
            printf("slot out of range\n");
            return 1;
        }
    }
    return 0;
}

int main()
{
    int cases = 0;
    const int tts[] = {1, 2, 3, 7, 196, 391};
    const int nps[] = {0, 1, 2, 5, 16, 40, 782};
    const int nss[] = {0, 1, 3, 40};
    const int Bs[] = {1, 2, 3, 7, 152, 304, 1000};
    for (int TT : tts)
        for (int np : nps)
            for (int ns : nss) {
                if (np + ns == 0) continue;
                for (int B : Bs) {
                    const long long units = (long long)TT * (np + ns);
                    const int Bu = (int)(B > units ? units : B);
                    for (int w = 0; w < 3; ++w) {
                        const int wp = w == 0 ? 1 : 10, wsg = w == 0 ? 1 : (w == 1 ? 28 : 20);
                        if (check(TT, np, ns, wp, wsg, Bu)) return 1;
                        ++cases;
                    }
                }
            }
    printf("OK %d cases\n", cases);
    return 0;
}
