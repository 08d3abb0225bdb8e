// Host harness for the Q0.64 angle quantiser of the pass scheduler: reads
// doubles (turns) from standard input, one per line, and prints the int64
// that the library stores for each (the angle mod 1 turn in units of 2^-64).
#include <cstdint>
#include <cstdio>
#include <string>

namespace sd {
int64_t turns_q64(double t);
void set_last_error(const std::string &) {}
}  // namespace sd

int main() {
    double t;
    while (std::scanf("%lf", &t) == 1) std::printf("%lld\n", (long long)sd::turns_q64(t));
    return 0;
}
