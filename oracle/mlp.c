/* placeholder: filled in with the MLP reference */
#include "oracle.h"
