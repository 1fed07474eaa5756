#include "rcb_internal.cuh"
namespace rcb {
int gravity_backward(rcb_tree *, const double *, const double *, double *, double *) { return RCB_ERR_STATE; }
}
