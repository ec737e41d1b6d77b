// placeholder, replaced by the tcgen05 transform kernels
#include "kernels.h"
namespace bx {
bool tc_supported() { return false; }
void launch_prec_tc(const LaunchCfg&, int, int, int) {}
}  // namespace bx
