// Host build of the float-float helpers (csrc/ff.cuh) for the CPU tests: reads operand
// pairs from stdin and prints the helpers' results as hexadecimal floats, which the test
// compares with exact rational arithmetic. The warp shuffle is not exercised here.
#include <cmath>
#include <cstdio>
#include <cstring>

#define __device__
#define __forceinline__ inline
#define __shfl_xor_sync(mask, v, o) (v)
#include "ff.cuh"

using rtp::ff;

int main() {
    char op[16];
    while (std::scanf("%15s", op) == 1) {
        if (!std::strcmp(op, "two_sum")) {
            float a, b;
            if (std::scanf("%a %a", &a, &b) != 2) return 1;
            const ff r = rtp::two_sum(a, b);
            std::printf("%a %a\n", r.hi, r.lo);
        } else if (!std::strcmp(op, "mul") || !std::strcmp(op, "add")) {
            ff x, y;
            if (std::scanf("%a %a %a %a", &x.hi, &x.lo, &y.hi, &y.lo) != 4) return 1;
            const ff r = op[0] == 'm' ? rtp::ff_mul(x, y) : rtp::ff_add(x, y);
            std::printf("%a %a\n", r.hi, r.lo);
        } else if (!std::strcmp(op, "recip") || !std::strcmp(op, "sqrt")) {
            ff x;
            if (std::scanf("%a %a", &x.hi, &x.lo) != 2) return 1;
            const ff r = op[0] == 'r' ? rtp::ff_recip(x) : rtp::ff_sqrt(x);
            std::printf("%a %a\n", r.hi, r.lo);
        } else if (!std::strcmp(op, "dot")) {   // n, then n pairs x_i y_i: sum x_i y_i
            int n;
            if (std::scanf("%d", &n) != 1) return 1;
            ff acc = {0.f, 0.f};
            for (int i = 0; i < n; ++i) {
                ff x, y;
                if (std::scanf("%a %a %a %a", &x.hi, &x.lo, &y.hi, &y.lo) != 4) return 1;
                rtp::ff_dot_acc(acc, x, y);
            }
            acc = rtp::ff_renorm(acc);
            std::printf("%a %a\n", acc.hi, acc.lo);
        } else if (!std::strcmp(op, "split")) {  // a double through ff and back
            double d;
            if (std::scanf("%la", &d) != 1) return 1;
            const ff r = rtp::ff_from_double(d);
            std::printf("%a %a %a\n", r.hi, r.lo, rtp::ff_to_double(r));
        }
    }
    return 0;
}
