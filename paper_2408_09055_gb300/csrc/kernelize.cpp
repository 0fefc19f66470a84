// Kernelize (Alg. 3 with the extensible-qubit reduction of Alg. 4).
#include "internal.hpp"

namespace qs {

int plan_kernelize(PlanImpl* p) {
  (void)p;
  return QS_EUNSUPPORTED;
}

}  // namespace qs
