/* placeholder: filled in with the multifluid dust oracle */
#include "oracle.h"
